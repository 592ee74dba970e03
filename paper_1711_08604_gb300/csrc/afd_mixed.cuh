// Mixed-radix Stockham transforms for N = 2^a 3^b 5^c 7^d 11^e 13^f (not a
// power of two) and the work-item bodies of the mixed-radix kernels, shared
// by the per-step kernels (afd_mixed.cu) and the multi-signal persistent
// kernel (afd_multi.cu).
#pragma once
#include <climits>
#include <cstdint>

#include "../../include/afd.h"
#include "afd_device.cuh"
#include "afd_fft.cuh"
#include "afd_internal.h"

namespace afd {

constexpr int MX_THREADS = 256;

// CTAs of the split forward transform: the largest power of two dividing N,
// at most 16, when the remaining N / S points need two or more passes; 1:
// one CTA per signal.
__host__ __device__ inline int mx_split(int N) {
  int S = N & -N;
  if (S > 16) S = 16;
  if (S < 2) return 1;
  int r[MIXED_MAX_PASSES];
  return mixed_schedule(N / S, r) >= 2 ? S : 1;
}

// X_k = sum_{q<3} v_q exp(DIR 2 pi i q k / 3)
template <int DIR, typename T>
__device__ __forceinline__ void dft3(V2<T>* v) {
  const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
  const V2<T> a = v[0], t1 = cadd<T>(v[1], v[2]), d = csub<T>(v[1], v[2]);
  const V2<T> m = mk2<T>(a.x - (T)0.5 * t1.x, a.y - (T)0.5 * t1.y);
  // DIR i h d
  const V2<T> r = DIR > 0 ? mk2<T>(-h * d.y, h * d.x) : mk2<T>(h * d.y, -h * d.x);
  v[0] = cadd<T>(a, t1);
  v[1] = cadd<T>(m, r);
  v[2] = csub<T>(m, r);
}

// X_k = sum_{q<5} v_q exp(DIR 2 pi i q k / 5), from the symmetric pairs
// t1 = v1 + v4, t2 = v2 + v3, t3 = v1 - v4, t4 = v2 - v3.
template <int DIR, typename T>
__device__ __forceinline__ void dft5(V2<T>* v) {
  const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
  const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
  const T s1 = (T)0.95105651629515357212;   // sin(2 pi / 5)
  const T s2 = (T)0.58778525229247312917;   // sin(4 pi / 5)
  const V2<T> v0 = v[0];
  const V2<T> t1 = cadd<T>(v[1], v[4]), t2 = cadd<T>(v[2], v[3]);
  const V2<T> t3 = csub<T>(v[1], v[4]), t4 = csub<T>(v[2], v[3]);
  const V2<T> A = mk2<T>(v0.x + c1 * t1.x + c2 * t2.x, v0.y + c1 * t1.y + c2 * t2.y);
  const V2<T> C = mk2<T>(v0.x + c2 * t1.x + c1 * t2.x, v0.y + c2 * t1.y + c1 * t2.y);
  // P = s1 t3 + s2 t4, Q = s2 t3 - s1 t4; the odd parts are DIR i P and DIR i Q
  const V2<T> P = mk2<T>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
  const V2<T> Q = mk2<T>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
  const V2<T> iP = DIR > 0 ? mk2<T>(-P.y, P.x) : mk2<T>(P.y, -P.x);
  const V2<T> iQ = DIR > 0 ? mk2<T>(-Q.y, Q.x) : mk2<T>(Q.y, -Q.x);
  v[0] = cadd<T>(v0, cadd<T>(t1, t2));
  v[1] = cadd<T>(A, iP);
  v[2] = cadd<T>(C, iQ);
  v[3] = csub<T>(C, iQ);
  v[4] = csub<T>(A, iP);
}

// X_k = sum_{q<R} v_q exp(DIR 2 pi i q k / R) for an odd prime R, from the
// symmetric pairs t_q = v_q + v_{R-q}, d_q = v_q - v_{R-q} (q = 1 .. H,
// H = (R - 1) / 2):
//   X_0 = v_0 + sum_q t_q,
//   X_k, X_{R-k} = v_0 + sum_q t_q cos(2 pi q k / R)  +-  DIR i sum_q d_q sin(2 pi q k / R).
// rc[m], rs[m] (m = 1 .. H) hold cos and sin of 2 pi m / R; (q k) mod R is a
// compile-time index once the loops are unrolled.
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_odd(V2<T>* v, const T* rc, const T* rs) {
  constexpr int H = (R - 1) / 2;
  V2<T> t[H + 1], d[H + 1];
  V2<T> x0 = v[0];
#pragma unroll
  for (int q = 1; q <= H; ++q) {
    t[q] = cadd<T>(v[q], v[R - q]);
    d[q] = csub<T>(v[q], v[R - q]);
    x0 = cadd<T>(x0, t[q]);
  }
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    V2<T> a = v[0], b = mk2<T>((T)0, (T)0);
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      const int m = (q * k) % R;  // cos and sin of 2 pi m / R from the first half
      const T c = m <= H ? rc[m] : rc[R - m];
      const T sn = m <= H ? rs[m] : -rs[R - m];
      a = mk2<T>(a.x + c * t[q].x, a.y + c * t[q].y);
      b = mk2<T>(b.x + sn * d[q].x, b.y + sn * d[q].y);
    }
    // DIR i b
    const V2<T> ib = DIR > 0 ? mk2<T>(-b.y, b.x) : mk2<T>(b.y, -b.x);
    v[k] = cadd<T>(a, ib);
    v[R - k] = csub<T>(a, ib);
  }
  v[0] = x0;
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_any(V2<T>* v, const T* rc, const T* rs) {
  if constexpr (R == 3) dft3<DIR, T>(v);
  else if constexpr (R == 5) dft5<DIR, T>(v);
  else if constexpr (R == 7 || R == 11 || R == 13) dft_odd<R, DIR, T>(v, rc, rs);
  else dft<R, DIR, T>(v);
}

// One Stockham pass of radix R; src(b, q, N/R) is input q of butterfly b,
// dst(i, value) takes output i.  tw: the N twiddles w^k, in shared memory
// (TWS) or in global memory (read through the read-only cache).
template <typename T, int R, int DIR, bool TWS, class Src, class Dst>
__device__ __forceinline__ void mx_pass(int N, int Ns, const V2<T>* __restrict__ tw, Src& src, Dst& dst) {
  const int NR = N / R, step = N / (Ns * R);
  // cos and sin of 2 pi m / R = w^(m N / R), m = 1 .. (R - 1) / 2, for the odd
  // prime radices that use dft_odd
  constexpr int H = R > 5 && (R & 1) ? (R - 1) / 2 : 0;
  T rc[H + 1], rs[H + 1];
#pragma unroll
  for (int m = 1; m <= H; ++m) {
    V2<T> w;
    if constexpr (TWS) w = tw[m * NR];
    else w = __ldg(&tw[m * NR]);
    rc[m] = w.x;
    rs[m] = w.y;
  }
  for (int b = threadIdx.x; b < NR; b += MX_THREADS) {
    const int k = b % Ns;
    V2<T> v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = src(b, q, NR);
    if (k != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        V2<T> w;  // q k step < N
        if constexpr (TWS) w = tw[q * k * step];
        else w = __ldg(&tw[q * k * step]);
        v[q] = DIR > 0 ? cmul<T>(v[q], w) : cmulc<T>(v[q], w);
      }
    }
    dft_any<R, DIR, T>(v, rc, rs);
    const int base = (b - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) dst(base + q * Ns, v[q]);
  }
}

template <typename T, int DIR, bool TWS, class Src, class Dst>
__device__ __forceinline__ void mx_pass_any(int R, int N, int Ns, const V2<T>* __restrict__ tw, Src& src,
                                            Dst& dst) {
  switch (R) {
    case 16: mx_pass<T, 16, DIR, TWS>(N, Ns, tw, src, dst); break;
    case 8: mx_pass<T, 8, DIR, TWS>(N, Ns, tw, src, dst); break;
    case 4: mx_pass<T, 4, DIR, TWS>(N, Ns, tw, src, dst); break;
    case 2: mx_pass<T, 2, DIR, TWS>(N, Ns, tw, src, dst); break;
    case 3: mx_pass<T, 3, DIR, TWS>(N, Ns, tw, src, dst); break;
    case 5: mx_pass<T, 5, DIR, TWS>(N, Ns, tw, src, dst); break;
    case 7: mx_pass<T, 7, DIR, TWS>(N, Ns, tw, src, dst); break;
    case 11: mx_pass<T, 11, DIR, TWS>(N, Ns, tw, src, dst); break;
    default: mx_pass<T, 13, DIR, TWS>(N, Ns, tw, src, dst); break;
  }
}

// The whole transform of N points with the np radices radix[] (at least two
// passes): first(b, q, N/R0) supplies pass 0's inputs, last(i, value)
// consumes the natural-order outputs.  tw: the N twiddles w^k of this
// length; buf holds 2 N points.  Every thread of the CTA must call it.
template <typename T, int DIR, bool TWS, class I, class First, class Last>
__device__ void mx_run_n(int N, int np, const I* radix, V2<T>* buf, const V2<T>* __restrict__ tw, First& first,
                         Last& last) {
  V2<T>* cur = buf;
  V2<T>* nxt = buf + N;
  auto to_cur = [&](int i, V2<T> x) { cur[i] = x; };
  mx_pass_any<T, DIR, TWS>(radix[0], N, 1, tw, first, to_cur);
  int Ns = radix[0];
  for (int ps = 1; ps < np; ++ps) {
    __syncthreads();
    const int R = radix[ps];
    auto from_cur = [&](int b, int q, int NR) { return cur[b + q * NR]; };
    if (ps + 1 < np) {
      auto to_nxt = [&](int i, V2<T> x) { nxt[i] = x; };
      mx_pass_any<T, DIR, TWS>(R, N, Ns, tw, from_cur, to_nxt);
      V2<T>* t = cur;
      cur = nxt;
      nxt = t;
    } else {
      mx_pass_any<T, DIR, TWS>(R, N, Ns, tw, from_cur, last);
    }
    Ns *= R;
  }
}
// ... of the plan's length N
template <typename T, int DIR, bool TWS, class First, class Last>
__device__ void mx_run(const PlanDev& p, V2<T>* buf, const V2<T>* __restrict__ tw, First& first, Last& last) {
  mx_run_n<T, DIR, TWS>(p.N, p.mix_npass, p.mix_radix, buf, tw, first, last);
}

template <typename T>
__device__ __forceinline__ const V2<T>* mx_twiddles(const PlanDev& p) {
  if constexpr (sizeof(T) == 4) return p.tw32n; else return p.tw64;
}

// Whether the N twiddles fit in shared memory after the two N-point buffers.
template <typename T>
__host__ __device__ constexpr bool mx_tw_fits(int N) {
  return 3 * (size_t)N * sizeof(V2<T>) <= (size_t)MIXED_MAX_SMEM;
}

// mx_run with the twiddles staged in shared memory (after buf's 2 N points)
// when they fit: each pass then reads them without a global-memory round
// trip.  Every thread of the CTA must call it.
template <typename T, int DIR, class First, class Last>
__device__ void mx_run_staged(const PlanDev& p, V2<T>* buf, First& first, Last& last) {
  const V2<T>* twg = mx_twiddles<T>(p);
  const int N = p.N;
  if (mx_tw_fits<T>(N)) {
    V2<T>* tws = buf + 2 * N;
    for (int i = threadIdx.x; i < N; i += MX_THREADS) tws[i] = __ldg(&twg[i]);
    __syncthreads();
    mx_run<T, DIR, true>(p, buf, tws, first, last);
  } else {
    mx_run<T, DIR, false>(p, buf, twg, first, last);
  }
}


// ------------------------------------------------------------ work items --
// The bodies of the mixed-radix kernels, shared with the multi-signal
// persistent kernel (MX_THREADS threads per CTA in both), which passes the
// work item's indices explicitly: the same values either way.

// Grid item: radius s of signal ids[sig], whose grid has `items` items; f(l) =
// r_s^l c_l / N, inverse transform, objective w_s^2 |F_s(j)|^2, the radius's
// best pair(s) and, in the signal's last item, the selection of Step 2.
// scr: the FP32 selection's scratch (unused in FP64).
template <typename T>
__device__ __forceinline__ void grid_mixed_body(const SlotDev* __restrict__ slots, const int* __restrict__ ids,
                                                int s, int sig, int items, SelectScratch* scr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  const SlotDev& sd = slots[ids[sig]];
  const int M = sd.p.M;
  const bool active = s < M;
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw);
  if constexpr (sizeof(T) == 4) {
    __shared__ Best2F red[32];
    Best2F best;
    best.init();
    if (active) {
      // f(l) = r_s^l c_l / N with r_s^l = lo[l mod B] hi[l div B], B = N / R0:
      // input q of butterfly b of pass 0 is l = b + q B
      const int B = sd.p.B, R0 = sd.p.mix_radix[0];
      const float* lo = sd.p.rlo32 + (size_t)s * B;
      const float* hi = sd.p.rhi32 + (size_t)s * R0;
      const float2* c = sd.c32;
      auto first = [&](int b, int q, int NR) {
        const float rp = __ldg(&lo[b]) * __ldg(&hi[q]);
        const float2 x = __ldcg(&c[b + q * NR]);
        return make_float2(x.x * rp, x.y * rp);
      };
      auto last = [&](int i, float2 x) { best.insert(norm2<float>(x), i); };
      mx_run_staged<float, +1>(sd.p, buf, first, last);
    }
    group_reduce<MX_THREADS>(best, red);
    if (threadIdx.x == 0 && active) {
      const float w2 = obj_w32(sd, s);
      Top2F o;
      o.v1 = best.v1 * w2;
      o.v2 = best.v2 * w2;
      o.j1 = best.j1;
      o.j2 = best.j2;
      reinterpret_cast<Top2F*>(sd.top2)[s] = o;
      if (o.v1 >= 0.0f && o.v1 <= 3.402823466e38f) atomicMax(&sd.ctl->vmax_bits, __float_as_uint(o.v1));
    }
    if (!arrive_last(&sd.ctl->cnt_grid, items, &s_last)) return;
    select_candidates_f32<MX_THREADS>(sd, sd.ctl->k, 1, *scr);
  } else {
    __shared__ Best1D red[32];
    Best1D best;
    best.init();
    if (active) {
      const int B = sd.p.B, R0 = sd.p.mix_radix[0];
      const double* lo = sd.p.rlo64 + (size_t)s * B;
      const double* hi = sd.p.rhi64 + (size_t)s * R0;
      const double2* c = sd.c64;
      auto first = [&](int b, int q, int NR) {
        const double rp = __ldg(&lo[b]) * __ldg(&hi[q]);
        const double2 x = __ldcg(&c[b + q * NR]);
        return make_double2(x.x * rp, x.y * rp);
      };
      auto last = [&](int i, double2 x) { best.insert(norm2<double>(x), i, x); };
      mx_run_staged<double, +1>(sd.p, buf, first, last);
    }
    group_reduce<MX_THREADS>(best, red);
    if (threadIdx.x == 0 && active) {
      const double w = sd.p.w64[s];
      Top2D o;
      o.v1 = best.v * (w * w) * obj_rho64(sd, s);
      o.j1 = best.j;
      o.f1 = best.f;
      o.v2 = -1.0;
      o.j2 = INT_MAX;
      o.f2 = make_double2(0.0, 0.0);
      reinterpret_cast<Top2D*>(sd.top2)[s] = o;
    }
    if (!arrive_last(&sd.ctl->cnt_grid, items, &s_last)) return;
    __syncthreads();
    select_best_f64<MX_THREADS>(sd, sd.ctl->k, red);
  }
}

// Forward item, one CTA per signal: c_l / N = (1/N) sum_m G(z_m) w^{-ml}.
template <typename T>
__device__ __forceinline__ void forward_mixed_body(const SlotDev* __restrict__ slots, const int* __restrict__ ids,
                                                   int sig) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SlotDev& sd = slots[ids[sig]];
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw);
  if constexpr (sizeof(T) == 4) {
    const float2* g = sd.g32;  // G / N in FP32, written by the update
    float2* c = sd.c32;
    auto first = [&](int b, int q, int NR) { return __ldcg(&g[b + q * NR]); };
    auto last = [&](int i, float2 x) { c[i] = x; };
    mx_run_staged<float, -1>(sd.p, buf, first, last);
  } else {
    const double2* G = sd.G;
    double2* c = sd.c64;
    const double n = (double)sd.p.N;
    auto first = [&](int b, int q, int NR) {
      const double2 x = __ldcg(&G[b + q * NR]);
      return make_double2(x.x / n, x.y / n);
    };
    auto last = [&](int i, double2 x) { c[i] = x; };
    mx_run_staged<double, -1>(sd.p, buf, first, last);
  }
}

// Forward item h of S (S = mx_split(N) > 1) of signal ids[sig]: one
// decimation-in-frequency step of radix S, the splitting of Theorem 2.1 with
// radix S.  With N' = N / S, l = l' + p N' and j = S j' + h,
//   c_j = sum_{l' < N'} w_{N'}^{-j' l'} [ w^{-h l'} sum_{p < S} x(l' + p N') e^{-2 pi i h p / S} ],
// so item h forms the bracket for its N' points l' and transforms it with the
// mixed-radix passes of N' (w_{N'}^k = w^{S k}), writing c_{S j' + h}.
template <typename T>
__device__ __forceinline__ void forward_mixed_split_body(const SlotDev* __restrict__ slots,
                                                         const int* __restrict__ ids, int h, int sig, int S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SlotDev& sd = slots[ids[sig]];
  const int N = sd.p.N, Np = N / S;
  int radix[MIXED_MAX_PASSES];
  const int np = mixed_schedule(Np, radix);
  V2<T>* buf = reinterpret_cast<V2<T>*>(smem_raw);
  V2<T>* tws = buf + 2 * Np;
  const V2<T>* twg = mx_twiddles<T>(sd.p);
  for (int i = threadIdx.x; i < Np; i += MX_THREADS) tws[i] = __ldg(&twg[(size_t)S * i]);
  // e^{-2 pi i h p / S} = conj(w^{((h p) mod S) N'}), p < S <= 16
  V2<T> ws[16];
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    if (p < S) {
      const V2<T> w = __ldg(&twg[(size_t)((h * p) % S) * Np]);
      ws[p] = mk2<T>(w.x, -w.y);
    }
  }
  __syncthreads();
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  const T n = (T)N;
  auto first = [&](int b, int q, int NR) {
    const int l = b + q * NR;
    V2<T> acc = mk2<T>((T)0, (T)0);
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      if (p < S) {
        V2<T> x;
        if constexpr (sizeof(T) == 4) {
          x = __ldcg(&sd.g32[l + p * Np]);  // G / N in FP32, written by the update
        } else {
          const double2 g = __ldcg(&sd.G[l + p * Np]);
          x = make_double2(g.x / n, g.y / n);
        }
        acc = cadd<T>(acc, cmul<T>(x, ws[p]));
      }
    }
    return cmulc<T>(acc, __ldg(&twg[h * l]));  // times w^{-h l'}; h l' < N
  };
  V2<T>* c;
  if constexpr (sizeof(T) == 4) c = sd.c32; else c = sd.c64;
  auto last = [&](int i, V2<T> x) { c[S * i + h] = x; };
  mx_run_n<T, -1, true>(Np, np, radix, buf, tws, first, last);
}

// Dynamic shared memory of the mixed-radix items of length N: two buffers and
// the twiddles when they fit (grid and one-CTA forward), or two buffers and
// the twiddles of N / S points (split forward).
inline size_t mixed_launch_smem(int N, int prec) {
  const bool f32 = prec == AFD_FP32_GUARDED;
  const bool tw = f32 ? mx_tw_fits<float>(N) : mx_tw_fits<double>(N);
  return (tw ? 3 : 2) * (size_t)N * (f32 ? 8 : 16);
}
inline size_t mixed_split_smem(int N, int prec) {
  return 3 * (size_t)(N / mx_split(N)) * (prec == AFD_FP32_GUARDED ? 8 : 16);
}

}  // namespace afd
