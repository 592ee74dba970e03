// Shared-memory-resident FFT building blocks for sm_103a.
//
// A length-N transform (N = 2^LOGN <= 16384) is done by one group of TPF
// threads, each holding P points in registers.  The passes follow the Stockham
// self-sorting scheme: a pass of radix R over sub-transforms of length Ns reads
// x[b + q N/R] (q = 0..R-1) for butterfly b, multiplies input q by the twiddle
// w^(q (b mod Ns) N/(Ns R)), does an R-point DFT in registers and writes output
// q to ((b div Ns) Ns R + (b mod Ns) + q Ns).  After the last pass the values
// are the DFT in natural order, so the caller knows each output's index
// without a permutation.  The first pass may read its input straight from
// global memory and the last pass may consume its outputs from registers,
// leaving (passes - 1) shared-memory round trips.
//
// Radix schedule (FftSchedule): one short pass of 2^(LOGN mod 4) first (if
// LOGN is not a multiple of 4), then radix-16 passes.  Shared memory is padded with one
// element per 16 (index i -> i + i/16), which makes the strided stores of the
// first passes bank-conflict free.
//
// This is the FFT structure of Theorem 2.1 (Sec. 3.1), which splits the sum
// of Eq. (rcl) into even and odd halves once; here the split is applied
// recursively with radix 16 instead of radix 2.
#pragma once
#include <cuda_runtime.h>

namespace afd {

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using V2 = typename Vec2<T>::type;

template <typename T> __device__ __forceinline__ V2<T> mk2(T x, T y) { V2<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ V2<T> cadd(V2<T> a, V2<T> b) { return mk2<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ V2<T> csub(V2<T> a, V2<T> b) { return mk2<T>(a.x - b.x, a.y - b.y); }

// FP32 products and fused multiply-adds with the rounding fixed in the
// source (no contraction left to the compiler), so that the paired FP32 path
// below, which does the same operations two lanes at a time, gives the same
// bits.  FP64 has no paired path and keeps the compiler's contraction.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return a * b; }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return a * b + c; }

// |a|^2 = fma(a.re, a.re, a.im * a.im)
template <typename T> __device__ __forceinline__ T norm2(V2<T> a) { return fma_rn(a.x, a.x, mul_rn(a.y, a.y)); }

// a * b: re = fma(a.re, b.re, a.im * (-b.im)), im = fma(a.re, b.im, a.im * b.re)
template <typename T> __device__ __forceinline__ V2<T> cmul(V2<T> a, V2<T> b) {
  return mk2<T>(fma_rn(a.x, b.x, mul_rn(a.y, -b.y)), fma_rn(a.x, b.y, mul_rn(a.y, b.x)));
}
// a * conj(b): re = fma(a.re, b.re, a.im * b.im), im = fma(a.im, b.re, a.re * (-b.im))
template <typename T> __device__ __forceinline__ V2<T> cmulc(V2<T> a, V2<T> b) {
  return mk2<T>(fma_rn(a.x, b.x, mul_rn(a.y, b.y)), fma_rn(a.y, b.x, mul_rn(a.x, -b.y)));
}

// a * exp(DIR 2 pi i idx / 16) for a compile-time-constant idx in [0, 8).
template <int DIR, typename T>
__device__ __forceinline__ V2<T> mul_w16(V2<T> a, int idx) {
  const T C1 = (T)0.92387953251128675613;  // cos(pi/8)
  const T S1 = (T)0.38268343236508977173;  // sin(pi/8)
  const T H = (T)0.70710678118654752440;   // cos(pi/4)
  switch (idx) {
    case 0: return a;
    case 4: return DIR > 0 ? mk2<T>(-a.y, a.x) : mk2<T>(a.y, -a.x);
    case 2: return DIR > 0 ? mk2<T>(mul_rn(a.x - a.y, H), mul_rn(a.x + a.y, H))
                           : mk2<T>(mul_rn(a.x + a.y, H), mul_rn(a.y - a.x, H));
    case 6: return DIR > 0 ? mk2<T>(mul_rn(a.x + a.y, -H), mul_rn(a.x - a.y, H))
                           : mk2<T>(mul_rn(a.y - a.x, H), mul_rn(a.x + a.y, -H));
    case 1: return cmul<T>(a, mk2<T>(C1, DIR > 0 ? S1 : -S1));
    case 3: return cmul<T>(a, mk2<T>(S1, DIR > 0 ? C1 : -C1));
    case 5: return cmul<T>(a, mk2<T>(-S1, DIR > 0 ? C1 : -C1));
    default: return cmul<T>(a, mk2<T>(-C1, DIR > 0 ? S1 : -S1));
  }
}

// In-register R-point DFT, natural order in and out:
// X_k = sum_q v_q exp(DIR 2 pi i q k / R), R in {2, 4, 8, 16}.
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft(V2<T>* v) {
  if constexpr (R == 2) {
    V2<T> t = v[0];
    v[0] = cadd<T>(t, v[1]);
    v[1] = csub<T>(t, v[1]);
  } else {
    V2<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    dft<R / 2, DIR, T>(e);
    dft<R / 2, DIR, T>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      V2<T> t = mul_w16<DIR, T>(o[k], k * (16 / R));
      v[k] = cadd<T>(e[k], t);
      v[k + R / 2] = csub<T>(e[k], t);
    }
  }
}

__device__ __forceinline__ int smem_pad(int i) { return i + (i >> 4); }

// Radix schedule of a 2^logn transform, shared by device code and the host
// code that builds the twiddle and power tables: pass 0 has radix
// 2^(logn mod 4) when logn is not a multiple of 4, every other pass radix 16.
struct FftSchedule {
  static __host__ __device__ constexpr int npass(int logn) { return logn / 4 + (logn % 4 ? 1 : 0); }
  static __host__ __device__ constexpr int radix(int logn, int p) {
    return (p == 0 && logn % 4) ? (1 << (logn % 4)) : 16;
  }
  // length of the sub-transforms that pass p combines
  static __host__ __device__ constexpr int ns(int logn, int p) {
    int n = 1;
    for (int i = 0; i < p; ++i) n *= radix(logn, i);
    return n;
  }
  // Stage twiddle table: pass p >= 1 owns (radix - 1) * ns entries at tw_off,
  // entry (q - 1) * ns + k holding exp(2 pi i q k / (ns * radix)), so that a
  // warp's consecutive butterflies read consecutive entries.
  static __host__ __device__ constexpr int tw_off(int logn, int p) {
    int o = 0;
    for (int i = 1; i < p; ++i) o += (radix(logn, i) - 1) * ns(logn, i);
    return o;
  }
  static __host__ __device__ constexpr int tw_size(int logn) { return tw_off(logn, npass(logn)); }
  // Power table split: r^l = lo[l mod B] * hi[l / B] with B = N / radix(0),
  // so the pass-0 inputs of one thread share lo and differ only in hi.
  static __host__ __device__ constexpr int pow_b(int logn) { return (1 << logn) / radix(logn, 0); }
};

// Compile-time shape of one transform.  PP: points per thread, 0 for the
// default (16; 32 for FP32 at N = 16384 to keep 512 threads); a multiple of
// the radix 16 otherwise.
template <typename T, int LOGN, int PP = 0>
struct FftShape {
  static constexpr int N = 1 << LOGN;
  static constexpr int P = LOGN < 4 ? N : (PP ? PP : ((sizeof(T) == 4 && LOGN >= 14) ? 32 : 16));
  static_assert(LOGN < 4 || (P % 16 == 0 && P <= N), "points per thread: a multiple of 16");
  static constexpr int TPF = N / P;                    // threads per transform
  static constexpr int NPASS = FftSchedule::npass(LOGN);
  static constexpr int SMEM = N + N / 16 + 1;          // padded elements per transform
  static __host__ __device__ constexpr int radix(int p) { return FftSchedule::radix(LOGN, p); }
  static __host__ __device__ constexpr int ns(int p) { return FftSchedule::ns(LOGN, p); }
};

// Twiddles of pass PASS applied to the thread's butterflies, then the DFTs.
// tw is the stage twiddle table of FftSchedule, in global memory (read through
// the read-only cache) or, with TW_SMEM, in shared memory.
template <typename T, int LOGN, int DIR, int PASS, bool TW_SMEM = false, int PP = 0>
__device__ __forceinline__ void fft_pass(V2<T>* v, int t, const V2<T>* __restrict__ tw) {
  using S = FftShape<T, LOGN, PP>;
  constexpr int R = S::radix(PASS), NS = S::ns(PASS), NB = S::P / R;
  constexpr int OFF = FftSchedule::tw_off(LOGN, PASS);
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if constexpr (NS > 1) {
      const int b = t + i * S::TPF;
      const int k = b & (NS - 1);
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const V2<T> w = TW_SMEM ? tw[OFF + (q - 1) * NS + k] : __ldg(&tw[OFF + (q - 1) * NS + k]);
        v[i * R + q] = DIR > 0 ? cmul<T>(v[i * R + q], w) : cmulc<T>(v[i * R + q], w);
      }
    }
    dft<R, DIR, T>(&v[i * R]);
  }
}

// Store the outputs of pass PASS to shared memory.  When the stride is a
// multiple of 16, smem_pad(base + q s) = smem_pad(base) + q (s + s / 16): one
// padded base per butterfly and constant offsets (no index arithmetic per
// element).
template <typename T, int LOGN, int PASS, int PP = 0>
__device__ __forceinline__ void fft_store(const V2<T>* v, int t, V2<T>* buf) {
  using S = FftShape<T, LOGN, PP>;
  constexpr int R = S::radix(PASS), NS = S::ns(PASS), NB = S::P / R;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = t + i * S::TPF;
    const int k = b & (NS - 1);
    const int base = (b - k) * R + k;
    if constexpr (NS % 16 == 0) {
      V2<T>* p = buf + smem_pad(base);
#pragma unroll
      for (int q = 0; q < R; ++q) p[q * (NS + NS / 16)] = v[i * R + q];
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) buf[smem_pad(base + q * NS)] = v[i * R + q];
    }
  }
}

// Load the inputs of pass PASS from shared memory (constant offsets from one
// padded base when the stride N / R is a multiple of 16, as in fft_store).
template <typename T, int LOGN, int PASS, int PP = 0>
__device__ __forceinline__ void fft_load(V2<T>* v, int t, const V2<T>* buf) {
  using S = FftShape<T, LOGN, PP>;
  constexpr int R = S::radix(PASS), NB = S::P / R, ST = S::N / R;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = t + i * S::TPF;
    if constexpr (ST % 16 == 0) {
      const V2<T>* p = buf + smem_pad(b);
#pragma unroll
      for (int q = 0; q < R; ++q) v[i * R + q] = p[q * (ST + ST / 16)];
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) v[i * R + q] = buf[smem_pad(b + q * ST)];
    }
  }
}

// Global index of the input held in register slot e before pass 0.
template <typename T, int LOGN, int PP = 0>
__device__ __forceinline__ int fft_in_index(int t, int e) {
  using S = FftShape<T, LOGN, PP>;
  constexpr int R = S::radix(0);
  return t + (e / R) * S::TPF + (e % R) * (S::N / R);
}

// Output index held in register slot e after the last pass.
template <typename T, int LOGN, int PP = 0>
__device__ __forceinline__ int fft_out_index(int t, int e) {
  using S = FftShape<T, LOGN, PP>;
  constexpr int LP = S::NPASS - 1;
  constexpr int R = S::radix(LP), NS = S::ns(LP);
  const int b = t + (e / R) * S::TPF;
  const int k = b & (NS - 1);
  return (b - k) * R + k + (e % R) * NS;
}

// Register slot of the u-th smallest output index of a thread after the last
// pass; that index is t + TPF u.
template <typename T, int LOGN, int PP = 0>
__host__ __device__ constexpr int fft_out_slot(int u) {
  using S = FftShape<T, LOGN, PP>;
  constexpr int R = S::radix(S::NPASS - 1), NB = S::P / R;
  return (u % NB) * R + u / NB;
}

// The exchange between passes synchronises the threads of one transform: a
// warp barrier when the TPF threads of a transform lie in one warp, else the
// CTA barrier, or with GS the named barrier 1 + g of transform group g (TPF
// threads), so that the groups of a CTA run their transforms independently.
template <typename T, int LOGN, int PP = 0, bool GS = false>
__device__ __forceinline__ void fft_sync() {
  constexpr int TPF = FftShape<T, LOGN, PP>::TPF;
  if constexpr (TPF <= 32) {
    __syncwarp();
  } else if constexpr (GS) {
    static_assert(TPF % 32 == 0, "whole warps per group");
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / TPF)), "n"(TPF) : "memory");
  } else {
    __syncthreads();
  }
}

// Runs passes PASS..NPASS-1; v holds the inputs of pass PASS.  Every thread of
// the CTA (with GS: of the transform group) must call this, as it
// synchronises with fft_sync, including threads whose transform is idle.
// When a transform fits in a warp (or with GS) nothing orders other warps'
// use of shared memory: a caller that reuses buf across transforms
// synchronises itself.
template <typename T, int LOGN, int DIR, int PASS = 0, bool TW_SMEM = false, int PP = 0, bool GS = false>
__device__ __forceinline__ void fft_run(V2<T>* v, int t, V2<T>* buf, const V2<T>* __restrict__ tw) {
  using S = FftShape<T, LOGN, PP>;
  fft_pass<T, LOGN, DIR, PASS, TW_SMEM, PP>(v, t, tw);
  if constexpr (PASS + 1 < S::NPASS) {
    fft_store<T, LOGN, PASS, PP>(v, t, buf);
    fft_sync<T, LOGN, PP, GS>();
    fft_load<T, LOGN, PASS + 1, PP>(v, t, buf);
    fft_sync<T, LOGN, PP, GS>();
    fft_run<T, LOGN, DIR, PASS + 1, TW_SMEM, PP, GS>(v, t, buf, tw);
  }
}


// ---------------------------------------------------------------------------
// Paired FP32 transforms (32 points per thread), sm_100-family f32x2 arithmetic.
//
// The same Stockham passes, radix schedule, twiddles and rounding as fft_run,
// but each thread works on two adjacent butterflies (2m, 2m+1) at once: X[j]
// holds the real parts of their input or output j (.x of butterfly 2m, .y of
// 2m+1) and Y[j] the imaginary parts, so that every add, multiply and fused
// multiply-add of the butterflies is one packed instruction (FADD2, FMUL2,
// FFMA2) for two lanes that would take two.  Per lane the operations are
// those of the scalar path (cmul, cmulc, mul_w16, dft), so the outputs are
// bitwise those of fft_run.  In pass p thread t holds the pairs
// m = t + i TPF, i < P / (2 R_p).  Shared memory holds the real and the
// imaginary parts in two arrays of NP floats, element e at fpad(e) (two
// padding words per 32), so that the pair (e, e+1) (e even) is one 64-bit
// access and a warp's accesses spread over the banks.  The stage twiddles
// come from the paired table: entry j of FftSchedule's table for even j,
// followed by entry j + 1, as (re_j, re_j+1, im_j, im_j+1).
template <int LOGN>
struct FftPShape {
  static constexpr int N = 1 << LOGN;
  static constexpr int P = 32;
  static constexpr int TPF = N / P;
  static constexpr int NPASS = FftSchedule::npass(LOGN);
  static constexpr int NP = N + N / 16;  // floats per component array (fpad(N - 1) < NP)
  static_assert(LOGN >= 5, "32 points per thread");
};
__device__ __forceinline__ int fpad(int e) { return e + ((e >> 5) << 1); }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// (X, Y) * (WX, WY) per lane as cmul; with DIR < 0 times the conjugate, as cmulc
template <int DIR>
__device__ __forceinline__ void cmul_p(float2& X, float2& Y, float2 WX, float2 WY) {
  const float2 x = X;
  if constexpr (DIR > 0) {
    X = fma2(x, WX, mul2(Y, neg2(WY)));
    Y = fma2(x, WY, mul2(Y, WX));
  } else {
    X = fma2(x, WX, mul2(Y, WY));
    Y = fma2(Y, WX, mul2(x, neg2(WY)));
  }
}

// mul_w16 per lane: (X, Y) * exp(DIR 2 pi i idx / 16), idx in [0, 8)
template <int DIR>
__device__ __forceinline__ void mul_w16_p(float2& X, float2& Y, int idx) {
  const float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f, H = 0.70710678118654752440f;
  const float2 x = X, y = Y;
  switch (idx) {
    case 0: return;
    case 4:
      if (DIR > 0) { X = neg2(y); Y = x; } else { X = y; Y = neg2(x); }
      return;
    case 2:
      if (DIR > 0) { X = mul2(sub2(x, y), dup2(H)); Y = mul2(add2(x, y), dup2(H)); }
      else { X = mul2(add2(x, y), dup2(H)); Y = mul2(sub2(y, x), dup2(H)); }
      return;
    case 6:
      if (DIR > 0) { X = mul2(add2(x, y), dup2(-H)); Y = mul2(sub2(x, y), dup2(H)); }
      else { X = mul2(sub2(y, x), dup2(H)); Y = mul2(add2(x, y), dup2(-H)); }
      return;
    case 1: cmul_p<1>(X, Y, dup2(C1), dup2(DIR > 0 ? S1 : -S1)); return;
    case 3: cmul_p<1>(X, Y, dup2(S1), dup2(DIR > 0 ? C1 : -C1)); return;
    case 5: cmul_p<1>(X, Y, dup2(-S1), dup2(DIR > 0 ? C1 : -C1)); return;
    default: cmul_p<1>(X, Y, dup2(-C1), dup2(DIR > 0 ? S1 : -S1)); return;
  }
}

// dft<R, DIR> per lane on (X, Y)
template <int R, int DIR>
__device__ __forceinline__ void dft_p(float2* X, float2* Y) {
  if constexpr (R == 2) {
    const float2 tx = X[0], ty = Y[0];
    X[0] = add2(tx, X[1]);
    Y[0] = add2(ty, Y[1]);
    X[1] = sub2(tx, X[1]);
    Y[1] = sub2(ty, Y[1]);
  } else {
    float2 ex[R / 2], ey[R / 2], ox[R / 2], oy[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      ex[i] = X[2 * i];
      ey[i] = Y[2 * i];
      ox[i] = X[2 * i + 1];
      oy[i] = Y[2 * i + 1];
    }
    dft_p<R / 2, DIR>(ex, ey);
    dft_p<R / 2, DIR>(ox, oy);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      mul_w16_p<DIR>(ox[k], oy[k], k * (16 / R));
      X[k] = add2(ex[k], ox[k]);
      Y[k] = add2(ey[k], oy[k]);
      X[k + R / 2] = sub2(ex[k], ox[k]);
      Y[k + R / 2] = sub2(ey[k], oy[k]);
    }
  }
}

// Twiddles of pass PASS, then the DFTs, for the thread's pairs.
template <int LOGN, int DIR, int PASS>
__device__ __forceinline__ void fftp_pass(float2* X, float2* Y, int t, const float4* __restrict__ twp) {
  using S = FftPShape<LOGN>;
  constexpr int R = FftSchedule::radix(LOGN, PASS), NS = FftSchedule::ns(LOGN, PASS), NPR = S::P / (2 * R);
  constexpr int OFF = FftSchedule::tw_off(LOGN, PASS);
#pragma unroll
  for (int i = 0; i < NPR; ++i) {
    if constexpr (NS > 1) {
      const int k = (2 * (t + i * S::TPF)) & (NS - 1);  // even: butterfly 2m + 1 has k + 1
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const float4 w = __ldg(&twp[(OFF + (q - 1) * NS + k) >> 1]);
        cmul_p<DIR>(X[i * R + q], Y[i * R + q], make_float2(w.x, w.y), make_float2(w.z, w.w));
      }
    }
    dft_p<R, DIR>(&X[i * R], &Y[i * R]);
  }
}

// Outputs of pass PASS to shared memory: butterfly b's output q goes to
// (b - k) R + k + q NS, k = b mod NS; for NS >= 2 the pair's two outputs are
// adjacent (one 64-bit store per component), for NS = 1 they are R apart.
template <int LOGN, int PASS>
__device__ __forceinline__ void fftp_store(const float2* X, const float2* Y, int t, float* re, float* im) {
  using S = FftPShape<LOGN>;
  constexpr int R = FftSchedule::radix(LOGN, PASS), NS = FftSchedule::ns(LOGN, PASS), NPR = S::P / (2 * R);
#pragma unroll
  for (int i = 0; i < NPR; ++i) {
    const int b = 2 * (t + i * S::TPF);
    if constexpr (NS == 1) {
      // a butterfly's outputs are consecutive here: store outputs q, q + 1 of
      // each of the two butterflies as one 64-bit pair
#pragma unroll
      for (int q = 0; q < R; q += 2) {
        *reinterpret_cast<float2*>(re + fpad(b * R + q)) = make_float2(X[i * R + q].x, X[i * R + q + 1].x);
        *reinterpret_cast<float2*>(im + fpad(b * R + q)) = make_float2(Y[i * R + q].x, Y[i * R + q + 1].x);
        *reinterpret_cast<float2*>(re + fpad(b * R + R + q)) = make_float2(X[i * R + q].y, X[i * R + q + 1].y);
        *reinterpret_cast<float2*>(im + fpad(b * R + R + q)) = make_float2(Y[i * R + q].y, Y[i * R + q + 1].y);
      }
    } else {
      const int k = b & (NS - 1);
      const int base = (b - k) * R + k;
      if constexpr (NS % 32 == 0) {
        // fpad(base + q NS) = fpad(base) + q (NS + NS / 16)
        float2* pr = reinterpret_cast<float2*>(re + fpad(base));
        float2* pi = reinterpret_cast<float2*>(im + fpad(base));
#pragma unroll
        for (int q = 0; q < R; ++q) {
          pr[q * (NS + NS / 16) / 2] = X[i * R + q];
          pi[q * (NS + NS / 16) / 2] = Y[i * R + q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
          *reinterpret_cast<float2*>(re + fpad(base + q * NS)) = X[i * R + q];
          *reinterpret_cast<float2*>(im + fpad(base + q * NS)) = Y[i * R + q];
        }
      }
    }
  }
}

// Inputs of pass PASS from shared memory: butterfly b reads b + q N / R; the
// pair's two inputs are adjacent.
template <int LOGN, int PASS>
__device__ __forceinline__ void fftp_load(float2* X, float2* Y, int t, const float* re, const float* im) {
  using S = FftPShape<LOGN>;
  constexpr int R = FftSchedule::radix(LOGN, PASS), NPR = S::P / (2 * R), ST = S::N / R;
#pragma unroll
  for (int i = 0; i < NPR; ++i) {
    const int b = 2 * (t + i * S::TPF);
    if constexpr (ST % 32 == 0) {
      // constant offsets: fpad(b + q ST) = fpad(b) + q (ST + ST / 16)
      const float2* pr = reinterpret_cast<const float2*>(re + fpad(b));
      const float2* pi = reinterpret_cast<const float2*>(im + fpad(b));
#pragma unroll
      for (int q = 0; q < R; ++q) {
        X[i * R + q] = pr[q * (ST + ST / 16) / 2];
        Y[i * R + q] = pi[q * (ST + ST / 16) / 2];
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        X[i * R + q] = *reinterpret_cast<const float2*>(re + fpad(b + q * ST));
        Y[i * R + q] = *reinterpret_cast<const float2*>(im + fpad(b + q * ST));
      }
    }
  }
}

// Input element of pair i, lane l, input q of pass 0 (the caller loads these)
template <int LOGN>
__host__ __device__ constexpr int fftp_in_index(int t, int i, int l, int q) {
  using S = FftPShape<LOGN>;
  return 2 * (t + i * S::TPF) + l + q * (S::N / FftSchedule::radix(LOGN, 0));
}
// Output element held in lane l of X[q], Y[q] after the last pass (one pair
// per thread): 2 t + l + q N / 16.  In increasing order: u = 2 q + l.
template <int LOGN>
__host__ __device__ constexpr int fftp_out_index(int t, int l, int q) {
  return 2 * t + l + q * ((1 << LOGN) / 16);
}

// When the first pass has radix 2 (LOGN = 4k + 1), the pass-0 butterflies
// b = m + q N/32 (q < 16) of thread m produce exactly the inputs q of its
// pass-1 pair (2m, 2m + 1): outputs 2b and 2b + 1.  So pass 0 runs in
// registers, without an exchange: a[q'] = x[m + q' N/32] (q' < 32) gives
// X[q] = (Re(a_q + a_q+16), Re(a_q - a_q+16)), Y[q] the imaginary parts, the
// additions of dft<2> lane for lane; fftp_run then starts at pass 1.
// (m = t: pass 1 has one pair per thread.)
template <int LOGN>
__host__ __device__ constexpr int fftp_r2_in_index(int t, int qq) {
  return t + qq * ((1 << LOGN) / 32);
}
__device__ __forceinline__ void fftp_r2_pass0(const float2* a, float2* X, float2* Y) {
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    X[q] = make_float2(a[q].x + a[q + 16].x, a[q].x - a[q + 16].x);
    Y[q] = make_float2(a[q].y + a[q + 16].y, a[q].y - a[q + 16].y);
  }
}

// Passes PASS..NPASS-1 on (X, Y); buf holds 2 NP floats (real parts, then
// imaginary parts).  Synchronisation as in fft_run (fft_sync with P = 32).
template <int LOGN, int DIR, int PASS = 0, bool GS = false>
__device__ __forceinline__ void fftp_run(float2* X, float2* Y, int t, float* buf, const float4* __restrict__ twp) {
  using S = FftPShape<LOGN>;
  static_assert(FftSchedule::radix(LOGN, S::NPASS - 1) == 16, "one pair per thread after the last pass");
  fftp_pass<LOGN, DIR, PASS>(X, Y, t, twp);
  if constexpr (PASS + 1 < S::NPASS) {
    fftp_store<LOGN, PASS>(X, Y, t, buf, buf + S::NP);
    fft_sync<float, LOGN, 32, GS>();
    fftp_load<LOGN, PASS + 1>(X, Y, t, buf, buf + S::NP);
    fft_sync<float, LOGN, 32, GS>();
    fftp_run<LOGN, DIR, PASS + 1, GS>(X, Y, t, buf, twp);
  }
}

}  // namespace afd
