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

#include "afd_fft.cuh"
#include "afd_internal.h"

namespace afd {

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ bool better_f(float va, int ja, float vb, int jb) {
  return va > vb || (va == vb && ja < jb);
}
__device__ __forceinline__ bool better_d(double va, int ja, double vb, int jb) {
  return va > vb || (va == vb && ja < jb);
}

struct Best2F {
  float v1, v2;
  int j1, j2;
  __device__ __forceinline__ void init() { v1 = v2 = -1.0f; j1 = j2 = INT_MAX; }
  __device__ __forceinline__ void insert(float v, int j) {
    if (better_f(v, j, v1, j1)) { v2 = v1; j2 = j1; v1 = v; j1 = j; }
    else if (better_f(v, j, v2, j2)) { v2 = v; j2 = j; }
  }
  __device__ __forceinline__ void merge(const Best2F& o) {
    if (better_f(o.v1, o.j1, v1, j1)) {
      if (better_f(v1, j1, o.v2, o.j2)) { v2 = v1; j2 = j1; } else { v2 = o.v2; j2 = o.j2; }
      v1 = o.v1; j1 = o.j1;
    } else if (better_f(o.v1, o.j1, v2, j2)) {
      v2 = o.v1; j2 = o.j1;
    }
  }
  __device__ __forceinline__ Best2F shfl(int off) const {
    Best2F r;
    r.v1 = __shfl_xor_sync(0xffffffffu, v1, off);
    r.v2 = __shfl_xor_sync(0xffffffffu, v2, off);
    r.j1 = __shfl_xor_sync(0xffffffffu, j1, off);
    r.j2 = __shfl_xor_sync(0xffffffffu, j2, off);
    return r;
  }
};

struct Best1D {
  double v;
  int j;
  double2 f;
  __device__ __forceinline__ void init() { v = -1.0; j = INT_MAX; f = make_double2(0.0, 0.0); }
  __device__ __forceinline__ void insert(double vv, int jj, double2 ff) {
    if (better_d(vv, jj, v, j)) { v = vv; j = jj; f = ff; }
  }
  __device__ __forceinline__ void merge(const Best1D& o) { insert(o.v, o.j, o.f); }
  __device__ __forceinline__ Best1D shfl(int off) const {
    Best1D r;
    r.v = __shfl_xor_sync(0xffffffffu, v, off);
    r.j = __shfl_xor_sync(0xffffffffu, j, off);
    r.f.x = __shfl_xor_sync(0xffffffffu, f.x, off);
    r.f.y = __shfl_xor_sync(0xffffffffu, f.y, off);
    return r;
  }
};

// Reduce B over each group of TPF consecutive threads; the group's thread
// t == 0 ends with the result.  All threads of the CTA must call it.
template <int TPF, class B>
__device__ __forceinline__ void group_reduce(B& b, B* red) {
  constexpr int W = TPF < 32 ? TPF : 32;
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) b.merge(b.shfl(off));
  if constexpr (TPF > 32) {
    constexpr int WPG = TPF / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = b;
    __syncthreads();
    if (lane == 0 && (warp % WPG) == 0) {
#pragma unroll 1
      for (int w = 1; w < WPG; ++w) b.merge(red[warp + w]);
    }
  }
}

// Deterministic FP64 block sum (fixed shuffle tree, warps added in order).
// Result valid in thread 0.
template <int THREADS>
__device__ __forceinline__ double block_sum(double x, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll 1
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
  }
  return s;
}

// Block-wide best (v, flat) over all threads; every thread gets the result.
template <int THREADS>
__device__ __forceinline__ void block_best_f(float& v, int& f, float* sv, int* sf) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, v, off);
    int of = __shfl_xor_sync(0xffffffffu, f, off);
    if (better_f(ov, of, v, f)) { v = ov; f = of; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { sv[warp] = v; sf[warp] = f; }
  __syncthreads();
  v = sv[0];
  f = sf[0];
#pragma unroll 1
  for (int w = 1; w < THREADS / 32; ++w)
    if (better_f(sv[w], sf[w], v, f)) { v = sv[w]; f = sf[w]; }
}

// Last-CTA detection: returns true in every thread of the CTA that is the
// last of `target` CTAs to arrive on *counter, and resets the counter.
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned target, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    *s_flag = (prev == target - 1u);
    if (*s_flag) *counter = 0u;
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ int ld_done(const SlotCtl* c) { return *((volatile const int*)&c->done); }

// ------------------------------------------------------------ grid kernel --

template <typename T, int LOGN>
struct GridCfg {
  using S = FftShape<T, LOGN>;
  static constexpr int FPC = S::TPF >= 256 ? 1 : 256 / S::TPF;  // transforms per CTA
  static constexpr int THREADS = S::TPF * FPC;
};

// FP32 selection in the last CTA of a signal: list the grid points whose
// objective is within tau of the largest one, best first, at most cap.
template <int THREADS>
__device__ void select_candidates_f32(const SlotDev& sd, int k) {
  __shared__ float sv[32];
  __shared__ int sf[32];
  const int M = sd.p.M, N = sd.p.N;
  const Top2F* top = reinterpret_cast<const Top2F*>(sd.top2);
  SlotCtl* ctl = sd.ctl;
  if (sd.force_a1_zero && k == 0) {
    if (threadIdx.x == 0) {
      sd.cand[0] = make_int2(0, 0);
      ctl->n_cand = 1;
      sd.rec[k].obj32 = __ldcg(&top[0].v1);
    }
    return;
  }
  float last_v = __int_as_float(0x7f800000);  // +inf: nothing chosen yet
  int last_f = -1;
  float thr = 0.0f;
  int n = 0;
#pragma unroll 1
  for (; n < sd.cap; ++n) {
    float bv = -1.0f;
    int bf = INT_MAX;
    for (int e = threadIdx.x; e < 2 * M; e += THREADS) {
      const int s = e >> 1;
      const float v = (e & 1) ? __ldcg(&top[s].v2) : __ldcg(&top[s].v1);
      const int j = (e & 1) ? __ldcg(&top[s].j2) : __ldcg(&top[s].j1);
      if (j == INT_MAX) continue;
      const int f = s * N + j;
      // strictly worse than the last pick, better than the current best
      if (better_f(last_v, last_f, v, f) && better_f(v, f, bv, bf)) { bv = v; bf = f; }
    }
    block_best_f<THREADS>(bv, bf, sv, sf);
    if (n == 0) {
      if (!(bv >= 0.0f) || bv == __int_as_float(0x7f800000)) break;  // nothing finite
      thr = bv - bv * (float)sd.tau;
      if (threadIdx.x == 0) sd.rec[k].obj32 = bv;
    }
    if (bf == INT_MAX || !(bv >= thr)) break;
    if (threadIdx.x == 0) sd.cand[n] = make_int2(bf / N, bf % N);
    last_v = bv;
    last_f = bf;
  }
  if (threadIdx.x == 0) {
    ctl->n_cand = n;
    if (n == sd.cap) ctl->err |= 1;  // the cap, not the window, ended the list
  }
}

// FP64 selection: global best of the per-radius maxima; writes the step record.
template <int THREADS>
__device__ void select_best_f64(const SlotDev& sd, int k, Best1D* red) {
  const int M = sd.p.M, N = sd.p.N;
  const Top2D* top = reinterpret_cast<const Top2D*>(sd.top2);
  Best1D b;
  b.init();
  if (sd.force_a1_zero && k == 0) {
    if (threadIdx.x == 0) {
      b.v = __ldcg(&top[0].v1);
      b.j = 0;  // radius 0: every angle ties, j1 == 0
      b.f.x = __ldcg(&top[0].f1.x);
      b.f.y = __ldcg(&top[0].f1.y);
    }
  } else {
    for (int s = threadIdx.x; s < M; s += THREADS) {
      const int j = __ldcg(&top[s].j1);
      if (j == INT_MAX) continue;
      double2 f;
      f.x = __ldcg(&top[s].f1.x);
      f.y = __ldcg(&top[s].f1.y);
      b.insert(__ldcg(&top[s].v1), s * N + j, f);
    }
    group_reduce<THREADS>(b, red);
  }
  if (threadIdx.x == 0) {
    StepRec& r = sd.rec[k];
    if (b.j == INT_MAX || !(b.v >= 0.0) || b.v > 1.79e308) {
      r.flags = 2;
      sd.ctl->err |= 2;
      sd.ctl->done = 1;
      r.s = -1;
      r.j = -1;
      return;
    }
    const int s = b.j / N, j = b.j % N;
    const double w = sd.p.w64[s];
    const double rr = sd.p.radii[s];
    const double2 z = sd.p.tw64[j];
    r.s = s;
    r.j = j;
    r.n_cand = 0;
    r.flags = 0;
    r.a_re = rr * z.x;
    r.a_im = rr * z.y;
    r.c_re = w * b.f.x;
    r.c_im = w * b.f.y;
    r.obj = r.c_re * r.c_re + r.c_im * r.c_im;
    r.obj32 = b.v;
  }
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(GridCfg<T, LOGN>::THREADS)
k_grid(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  using S = FftShape<T, LOGN>;
  using C = GridCfg<T, LOGN>;
  constexpr int N = S::N, P = S::P, TPF = S::TPF, FPC = C::FPC, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  const SlotDev& sd = slots[ids[blockIdx.y]];
  if (ld_done(sd.ctl)) return;

  const int g = threadIdx.x / TPF, t = threadIdx.x % TPF;
  const int s = blockIdx.x * FPC + g;
  const int M = sd.p.M;
  const bool active = s < M;
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw) + g * S::SMEM;

  // Pass-0 input f(l) = r_s^l c_l / N, read straight from the spectrum.
  V2<T> v[P];
  const V2<T>* tw;
  if constexpr (sizeof(T) == 4) tw = sd.p.tw32; else tw = sd.p.tw64;
  if (active) {
    const int B = sd.p.B;
    const int lb = 31 - __clz(B);
    const T* lo;
    const T* hi;
    const V2<T>* c;
    if constexpr (sizeof(T) == 4) {
      lo = sd.p.rlo32 + (size_t)s * B;
      hi = sd.p.rhi32 + (size_t)s * (N >> lb);
      c = sd.c32;
    } else {
      lo = sd.p.rlo64 + (size_t)s * B;
      hi = sd.p.rhi64 + (size_t)s * (N >> lb);
      c = sd.c64;
    }
#pragma unroll
    for (int e = 0; e < P; ++e) {
      const int l = fft_in_index<T, LOGN>(t, e);
      const T rp = __ldg(&hi[l >> lb]) * __ldg(&lo[l & (B - 1)]);
      const V2<T> x = __ldg(&c[l]);
      v[e] = mk2<T>(x.x * rp, x.y * rp);
    }
  } else {
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = mk2<T>((T)0, (T)0);
  }

  fft_run<T, LOGN, +1>(v, t, buf, tw);

  // Objective and per-radius best, straight from registers.
  if constexpr (sizeof(T) == 4) {
    __shared__ Best2F red[32];
    Best2F b;
    b.init();
#pragma unroll
    for (int e = 0; e < P; ++e) b.insert(v[e].x * v[e].x + v[e].y * v[e].y, fft_out_index<T, LOGN>(t, e));
    group_reduce<TPF>(b, red);
    if (t == 0 && active) {
      const float w2 = sd.p.wsq32[s];
      Top2F o;
      o.v1 = b.v1 * w2;
      o.v2 = b.v2 * w2;
      o.j1 = b.j1;
      o.j2 = b.j2;
      reinterpret_cast<Top2F*>(sd.top2)[s] = o;
    }
    if (!arrive_last(&sd.ctl->cnt_grid, gridDim.x, &s_last)) return;
    select_candidates_f32<THREADS>(sd, sd.ctl->k);
  } else {
    __shared__ Best1D red[32];
    Best1D b;
    b.init();
#pragma unroll
    for (int e = 0; e < P; ++e) b.insert(v[e].x * v[e].x + v[e].y * v[e].y, fft_out_index<T, LOGN>(t, e), v[e]);
    group_reduce<TPF>(b, red);
    if (t == 0 && active) {
      const double w = sd.p.w64[s];
      Top2D o;
      o.v1 = b.v * (w * w);
      o.j1 = b.j;
      o.f1 = b.f;
      o.v2 = -1.0;
      o.j2 = INT_MAX;
      o.f2 = make_double2(0.0, 0.0);
      reinterpret_cast<Top2D*>(sd.top2)[s] = o;
    }
    if (!arrive_last(&sd.ctl->cnt_grid, gridDim.x, &s_last)) return;
    __syncthreads();
    select_best_f64<THREADS>(sd, sd.ctl->k, red);
  }
}

// ----------------------------------------------------------- guard kernel --

// <G, e_a>~ partial sums over one chunk of samples for candidate a = r w^j:
// sum_m G(z_m) / (1 - r w^{j-m}), the kernel written as
// (1 - r cos + i r sin) / ((1 - r cos)^2 + (r sin)^2) to avoid cancellation.
__global__ void __launch_bounds__(FP64_THREADS)
k_guard(const SlotDev* __restrict__ slots, const int* __restrict__ ids, int cap) {
  __shared__ double red[FP64_THREADS / 32];
  __shared__ int s_last;
  const SlotDev& sd = slots[ids[blockIdx.y]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const int N = sd.p.N;
  const int Pg = chunks_of(N);
  const int cidx = blockIdx.x / Pg, p = blockIdx.x % Pg;
  const int n_cand = ctl->n_cand;
  if (cidx < n_cand) {
    const int2 cj = sd.cand[cidx];
    const double r = sd.p.radii[cj.x];
    const int j = cj.y;
    const int m0 = p * (N / Pg), m1 = m0 + N / Pg;
    double ar = 0.0, ai = 0.0;
    for (int m = m0 + threadIdx.x; m < m1; m += FP64_THREADS) {
      const double2 w = __ldg(&sd.p.tw64[(j - m) & (N - 1)]);
      const double u = fma(-r, w.x, 1.0);
      const double vv = r * w.y;
      const double inv = 1.0 / fma(u, u, vv * vv);
      const double kr = u * inv, ki = vv * inv;
      const double2 gm = sd.G[m];
      ar = fma(gm.x, kr, fma(-gm.y, ki, ar));
      ai = fma(gm.x, ki, fma(gm.y, kr, ai));
    }
    const double sr = block_sum<FP64_THREADS>(ar, red);
    const double si = block_sum<FP64_THREADS>(ai, red);
    if (threadIdx.x == 0) sd.gpart[cidx * Pg + p] = make_double2(sr, si);
  }
  if (!arrive_last(&ctl->cnt_guard, gridDim.x, &s_last)) return;
  // Candidate c's partial sums are added in chunk order by thread c.
  __shared__ double s_re[MAX_CAP], s_im[MAX_CAP], s_v[MAX_CAP];
  if (threadIdx.x < n_cand) {
    const int c = threadIdx.x;
    const int2 cj = sd.cand[c];
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < Pg; ++q) {
      const double2 pp = __ldcg(&sd.gpart[c * Pg + q]);
      sr += pp.x;
      si += pp.y;
    }
    const double sc = sd.p.sq64[cj.x] / (double)N;
    s_re[c] = sc * sr;
    s_im[c] = sc * si;
    s_v[c] = s_re[c] * s_re[c] + s_im[c] * s_im[c];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int k = ctl->k;
  StepRec& rec = sd.rec[k];
  int bs = -1, bj = -1;
  double bv = -1.0, bre = 0.0, bim = 0.0;
  for (int c = 0; c < n_cand; ++c) {
    const int2 cj = sd.cand[c];
    const double v = s_v[c];
    const int f = cj.x * N + cj.y, bf = bs * N + bj;
    if (bs < 0 || v > bv || (v == bv && f < bf)) {
      bs = cj.x; bj = cj.y; bv = v; bre = s_re[c]; bim = s_im[c];
    }
  }
  if (bs < 0 || !(bv <= 1.79e308)) {
    rec.s = -1;
    rec.j = -1;
    rec.flags = 2;
    ctl->err |= 2;
    ctl->done = 1;
    return;
  }
  const double rr = sd.p.radii[bs];
  const double2 z = sd.p.tw64[bj];
  rec.s = bs;
  rec.j = bj;
  rec.n_cand = n_cand;
  rec.flags = ctl->err & 1;
  rec.a_re = rr * z.x;
  rec.a_im = rr * z.y;
  rec.c_re = bre;
  rec.c_im = bim;
  rec.obj = bv;
}

// ---------------------------------------------------------- update kernel --

template <bool INIT>
__global__ void __launch_bounds__(FP64_THREADS)
k_update(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  __shared__ double red[FP64_THREADS / 32];
  __shared__ int s_last;
  const SlotDev& sd = slots[ids[blockIdx.y]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const int N = sd.p.N;
  const int Pu = chunks_of(N);
  const int p = blockIdx.x;
  const int m0 = p * (N / Pu), m1 = m0 + N / Pu;
  const int k = ctl->k;
  double e = 0.0;
  if constexpr (INIT) {
    for (int m = m0 + threadIdx.x; m < m1; m += FP64_THREADS) {
      const double2 g = sd.G[m];
      e = fma(g.x, g.x, fma(g.y, g.y, e));
    }
  } else {
    const StepRec& rec = sd.rec[k];
    const double ar = rec.a_re, ai = rec.a_im;
    const double na = sd.p.sq64[rec.s];  // sqrt(1 - |a|^2) with |a| = r_s
    const double cr = rec.c_re * na, ci = rec.c_im * na;
    for (int m = m0 + threadIdx.x; m < m1; m += FP64_THREADS) {
      const double2 z = __ldg(&sd.p.tw64[m]);
      const double2 g = sd.G[m];
      // u = 1 - conj(a) z
      const double ur = fma(-ar, z.x, fma(-ai, z.y, 1.0));
      const double ui = fma(ai, z.x, -ar * z.y);
      // numerator G u - c sqrt(1-|a|^2)
      const double nr = fma(g.x, ur, fma(-g.y, ui, -cr));
      const double ni = fma(g.x, ui, fma(g.y, ur, -ci));
      // divide by d = z - a
      const double dr = z.x - ar, di = z.y - ai;
      const double inv = 1.0 / fma(dr, dr, di * di);
      const double gr = fma(nr, dr, ni * di) * inv;
      const double gi = fma(ni, dr, -nr * di) * inv;
      sd.G[m] = make_double2(gr, gi);
      e = fma(gr, gr, fma(gi, gi, e));
    }
  }
  const double es = block_sum<FP64_THREADS>(e, red);
  if (threadIdx.x == 0) sd.epart[p] = es;
  if (!arrive_last(&ctl->cnt_update, gridDim.x, &s_last)) return;
  __shared__ double s_part[FP64_THREADS];
  for (int q = threadIdx.x; q < Pu; q += FP64_THREADS) s_part[q] = __ldcg(&sd.epart[q]);
  __syncthreads();
  if (threadIdx.x != 0) return;
  double E = 0.0;
  for (int q = 0; q < Pu; ++q) E += s_part[q];
  E /= (double)N;
  if constexpr (INIT) {
    ctl->E1 = E;
  } else {
    StepRec& rec = sd.rec[k];
    const double delta = ctl->E1 > 0.0 ? E / ctl->E1 : 0.0;
    rec.energy = E;
    rec.delta = delta;
    ctl->k = k + 1;
    if (k + 1 >= sd.K_max || (sd.tol > 0.0 && delta <= sd.tol)) ctl->done = 1;
  }
}

// --------------------------------------------------------- forward kernel --

template <typename T, int LOGN>
__global__ void __launch_bounds__(FftShape<T, LOGN>::TPF)
k_forward(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  using S = FftShape<T, LOGN>;
  constexpr int P = S::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SlotDev& sd = slots[ids[blockIdx.x]];
  if (ld_done(sd.ctl)) return;
  const int t = threadIdx.x;
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw);
  const double scale = 1.0 / (double)S::N;  // exact: N is a power of two
  V2<T> v[P];
#pragma unroll
  for (int e = 0; e < P; ++e) {
    const double2 g = sd.G[fft_in_index<T, LOGN>(t, e)];
    v[e] = mk2<T>((T)(g.x * scale), (T)(g.y * scale));
  }
  const V2<T>* tw;
  if constexpr (sizeof(T) == 4) tw = sd.p.tw32; else tw = sd.p.tw64;
  fft_run<T, LOGN, -1>(v, t, buf, tw);
  V2<T>* c;
  if constexpr (sizeof(T) == 4) c = sd.c32; else c = sd.c64;
#pragma unroll
  for (int e = 0; e < P; ++e) c[fft_out_index<T, LOGN>(t, e)] = v[e];
}

// --------------------------------------------------------------- launchers --

namespace {

template <typename T, int LOGN>
size_t grid_smem() {
  using S = FftShape<T, LOGN>;
  return sizeof(V2<T>) * (size_t)S::SMEM * GridCfg<T, LOGN>::FPC;
}
template <typename T, int LOGN>
size_t fwd_smem() {
  using S = FftShape<T, LOGN>;
  return sizeof(V2<T>) * (size_t)S::SMEM;
}

template <typename T, int LOGN>
cudaError_t grid_launch(const SlotDev* slots, const int* ids, int n, int Mmax, cudaStream_t st) {
  using C = GridCfg<T, LOGN>;
  dim3 grid((Mmax + C::FPC - 1) / C::FPC, n);
  k_grid<T, LOGN><<<grid, C::THREADS, grid_smem<T, LOGN>(), st>>>(slots, ids);
  return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t fwd_launch(const SlotDev* slots, const int* ids, int n, cudaStream_t st) {
  k_forward<T, LOGN><<<n, FftShape<T, LOGN>::TPF, fwd_smem<T, LOGN>(), st>>>(slots, ids);
  return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_grid<T, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)grid_smem<T, LOGN>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_forward<T, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fwd_smem<T, LOGN>());
}

#define AFD_FOR_EACH_LOGN(X) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)

}  // namespace

cudaError_t configure_kernels() {
  cudaError_t e = cudaSuccess;
#define X(L)                                             \
  if ((e = set_attrs<float, L>()) != cudaSuccess) return e; \
  if ((e = set_attrs<double, L>()) != cudaSuccess) return e;
  AFD_FOR_EACH_LOGN(X)
#undef X
  return set_attrs<float, 14>();
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

cudaError_t launch_grid(const SlotDev* slots, const int* ids, int n, int logN, int prec, int Mmax,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  switch (logN) {
#define X(L)                                                                          \
  case L:                                                                             \
    return prec ? grid_launch<float, L>(slots, ids, n, Mmax, st)                      \
                : grid_launch<double, L>(slots, ids, n, Mmax, st);
    AFD_FOR_EACH_LOGN(X)
#undef X
    case 14:
      if (prec) return grid_launch<float, 14>(slots, ids, n, Mmax, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
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
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_guard(const SlotDev* slots, const int* ids, int n, int logN, int cap, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(cap * chunks_of(1 << logN), n);
  k_guard<<<grid, FP64_THREADS, 0, st>>>(slots, ids, cap);
  return cudaGetLastError();
}

cudaError_t launch_update(const SlotDev* slots, const int* ids, int n, int logN, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(chunks_of(1 << logN), n);
  k_update<false><<<grid, FP64_THREADS, 0, st>>>(slots, ids);
  return cudaGetLastError();
}

cudaError_t launch_init(const SlotDev* slots, const int* ids, int n, int logN, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(chunks_of(1 << logN), n);
  k_update<true><<<grid, FP64_THREADS, 0, st>>>(slots, ids);
  return cudaGetLastError();
}

}  // namespace afd
