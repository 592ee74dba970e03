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
// a * b
template <typename T> __device__ __forceinline__ V2<T> cmul(V2<T> a, V2<T> b) {
  return mk2<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ V2<T> cmulc(V2<T> a, V2<T> b) {
  return mk2<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
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
    case 2: return DIR > 0 ? mk2<T>((a.x - a.y) * H, (a.x + a.y) * H)
                           : mk2<T>((a.x + a.y) * H, (a.y - a.x) * H);
    case 6: return DIR > 0 ? mk2<T>(-(a.x + a.y) * H, (a.x - a.y) * H)
                           : mk2<T>((a.y - a.x) * H, -(a.x + a.y) * H);
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

}  // namespace afd
