// Core AFD on non-uniform samples (the remark after Step 2 of the algorithm of
// Sec. 3.2: non-uniform sampling is handled by non-uniform DFTs), sm_103a.
//
// The signal is known at z_m = exp(i theta_m), m < nN, with quadrature
// weights w_m of dt / 2 pi; the rectangle rule of Eq. (formula1) becomes
//   <G, e_a>~ = sqrt(1 - |a|^2) sum_m w_m G(z_m) / (1 - a conj(z_m)).
// The grid keeps N equispaced angles, a_{s,j} = r_s w^j, w = exp(2 pi i / N).
// Expanding 1 / (1 - a conj(z)) = sum_l a^l conj(z)^l,
//   <G, e_a>~ = sqrt(1 - r_s^2) sum_{l >= 0} r_s^l w^{jl} c_l,
//   c_l = sum_m w_m G(z_m) exp(-i l theta_m)           (a non-uniform DFT),
// and folding l = l' + p N (w^{jN} = 1) gives an N-point inverse DFT of
//   f_s(l') = r_s^{l'} sum_p (r_s^N)^p c_{l' + p N},
// summed over the folds p < P_s with r_s^{P_s N} <= 2^-64 (the rest of the
// series is below FP64 resolution).  For equispaced samples c_l is periodic
// and the fold sum is the geometric factor 1 / (1 - r^N) of Eq. (rcl).
//
// Kernels of one step (FP32 grid, FP64 guard, remainder and energy):
//   k_nudft     c_l, l < Lc = max_s P_s x N, from w_m G(z_m) in FP32; the phase
//               l theta_m / 2 pi is formed exactly in 64-bit fixed point;
//   k_grid_nu   per radius the folded input, inverse FFT (the resident
//               Stockham transform of afd_fft.cuh), objective
//               (1 - r_s^2) |F_s(j)|^2, best pairs, last-CTA candidates;
//   k_guard_nu  the FP64 weighted rectangle rule at every candidate;
//   k_update_nu the Blaschke update of Sec. 2 at the samples, the weighted
//               energy sum_m w_m |G|^2, delta and the stop rule.
#include <climits>
#include <cstdint>

#include "../../include/afd.h"
#include "afd_device.cuh"
#include "afd_fft.cuh"
#include "afd_internal.h"

namespace afd {

namespace {

// l values per CTA and threads per CTA of the non-uniform DFT.  A step's DFT
// has only Lc (a few thousand) outputs: short blocks of l give enough CTAs to
// fill the GPU, and every thread walks its share of the samples.
constexpr int NUDFT_L = 8, NUDFT_THREADS = 256;

template <int LOGN>
struct NuCfg {
  using S = FftShape<float, LOGN>;
  static constexpr int FPC = S::TPF >= 256 ? 1 : 256 / S::TPF;  // radii per CTA
  static constexpr int THREADS = S::TPF * FPC;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)S::SMEM * FPC;
};

// c_l = sum_m w_m G(z_m) exp(-i l theta_m) for l < Lc.  CTA: NUDFT_L
// consecutive l = l0 + i; thread t takes the samples m = t, t + NUDFT_THREADS,
// ...  For each sample, exp(-i lc theta_m) at the block's middle lc = l0 +
// NUDFT_L / 2 comes from the exact 64-bit fixed-point phase lc theta_m / 2 pi,
// and the other powers from multiplying by exp(-+i theta_m) (at most
// NUDFT_L / 2 products), whose phase keeps 48 bits (a first-order correction
// of the 24-bit angle): one pair of sincospif per sample and block, not per
// term.
// Sums: each thread's partials, a shuffle tree in each warp, the warps in
// order.
__global__ void __launch_bounds__(NUDFT_THREADS)
k_nudft(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  __shared__ float2 part[NUDFT_THREADS / 32][NUDFT_L];
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[0]];
  pdl_wait();
  if (ld_done(sd.ctl)) return;
  const int l0 = blockIdx.x * NUDFT_L;
  const int n = sd.p.nN;
  constexpr int H = NUDFT_L / 2;
  const unsigned long long ulc = (unsigned long long)(l0 + H);
  constexpr float TWO_M24 = 5.9604644775390625e-8f;  // 2^-24
  constexpr float TWO_PI_M48 = 2.2322566310269275e-14f;  // 2 pi 2^-48
  float2 acc[NUDFT_L];
#pragma unroll
  for (int i = 0; i < NUDFT_L; ++i) acc[i] = make_float2(0.f, 0.f);
  for (int m = threadIdx.x; m < n; m += NUDFT_THREADS) {
    const unsigned long long u = __ldg(&sd.p.nU[m]);
    // exp(-i lc theta_m): the top 24 bits of the phase fraction (error below
    // 2 pi 2^-25)
    float s0, c0;
    sincospif(2.0f * ((float)((ulc * u) >> 40) * TWO_M24), &s0, &c0);
    // exp(-i theta_m): the top 24 bits, then a rotation by the next 24 bits'
    // angle d < 2 pi 2^-24 (cos d = 1 and sin d = d to FP32 precision)
    float s1, c1;
    sincospif(2.0f * ((float)(u >> 40) * TWO_M24), &s1, &c1);
    const float d = (float)((u >> 16) & 0xffffffull) * TWO_PI_M48;
    const float zr = fmaf(-s1, d, c1), zi = -fmaf(c1, d, s1);  // (c1 - i s1)(1 - i d)
    const float2 g = __ldcg(&sd.g32[m]);  // w_m G(z_m)
    // g exp(-i l theta_m) into acc[l - l0]: l = lc, then upwards (times
    // exp(-i theta_m)) and downwards (times its conjugate)
    float fr = c0, fi = -s0, br = c0, bi = -s0;
    acc[H].x = fmaf(g.x, fr, fmaf(-g.y, fi, acc[H].x));
    acc[H].y = fmaf(g.x, fi, fmaf(g.y, fr, acc[H].y));
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      if (k < H) {
        const float nr = fmaf(fr, zr, -fi * zi), ni = fmaf(fr, zi, fi * zr);
        fr = nr;
        fi = ni;
        acc[H + k].x = fmaf(g.x, fr, fmaf(-g.y, fi, acc[H + k].x));
        acc[H + k].y = fmaf(g.x, fi, fmaf(g.y, fr, acc[H + k].y));
      }
      const float nr = fmaf(br, zr, bi * zi), ni = fmaf(bi, zr, -br * zi);  // times conj(z)
      br = nr;
      bi = ni;
      acc[H - k].x = fmaf(g.x, br, fmaf(-g.y, bi, acc[H - k].x));
      acc[H - k].y = fmaf(g.x, bi, fmaf(g.y, br, acc[H - k].y));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NUDFT_L; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc[i].x += __shfl_xor_sync(0xffffffffu, acc[i].x, off);
      acc[i].y += __shfl_xor_sync(0xffffffffu, acc[i].y, off);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NUDFT_L; ++i) part[warp][i] = acc[i];
  }
  __syncthreads();
  if (threadIdx.x < NUDFT_L && l0 + (int)threadIdx.x < sd.p.nLc) {
    float2 r = part[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < NUDFT_THREADS / 32; ++w) {
      r.x += part[w][threadIdx.x].x;
      r.y += part[w][threadIdx.x].y;
    }
    sd.c32[l0 + threadIdx.x] = r;
  }
}

// One inverse transform per radius of the folded input; the rest as k_grid.
template <int LOGN>
__global__ void __launch_bounds__(NuCfg<LOGN>::THREADS)
k_grid_nu(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  using S = FftShape<float, LOGN>;
  using C = NuCfg<LOGN>;
  constexpr int N = S::N, P = S::P, TPF = S::TPF, FPC = C::FPC, THREADS = C::THREADS;
  constexpr int R0 = S::radix(0), B = FftSchedule::pow_b(LOGN), NB0 = P / R0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_last;
  __shared__ Best2F red[32];
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[blockIdx.y]];
  const int g = threadIdx.x / TPF, t = threadIdx.x % TPF;
  const int s = blockIdx.x * FPC + g;
  const int M = sd.p.M;
  const bool active = s < M;
  float2* buf = reinterpret_cast<float2*>(smem_raw) + g * S::SMEM;
  float2 v[P];
  if (active) {
    float h[R0], lb[NB0];
#pragma unroll
    for (int q = 0; q < R0; ++q) h[q] = __ldg(&sd.p.rhi32[(size_t)s * R0 + q]);
#pragma unroll
    for (int i = 0; i < NB0; ++i) lb[i] = __ldg(&sd.p.rlo32[(size_t)s * B + t + i * TPF]);
    const float rN = __ldg(&sd.p.nrN32[s]);
    const int folds = __ldg(&sd.p.nP[s]);
    pdl_wait();
    if (ld_done(sd.ctl)) return;
    const float2* c = sd.c32;
#pragma unroll
    for (int i = 0; i < NB0; ++i) {
#pragma unroll
      for (int q = 0; q < R0; ++q) {
        const int l = t + i * TPF + q * B;
        // sum_p (r^N)^p c_{l + p N}, Horner from the last fold
        float2 acc = __ldcg(&c[l + (folds - 1) * N]);
        for (int p = folds - 2; p >= 0; --p) {
          const float2 x = __ldcg(&c[l + p * N]);
          acc = make_float2(fmaf(acc.x, rN, x.x), fmaf(acc.y, rN, x.y));
        }
        const float rp = lb[i] * h[q];
        v[i * R0 + q] = make_float2(acc.x * rp, acc.y * rp);
      }
    }
  } else {
    pdl_wait();
    if (ld_done(sd.ctl)) return;
#pragma unroll
    for (int e = 0; e < P; ++e) v[e] = make_float2(0.f, 0.f);
  }
  fft_run<float, LOGN, +1>(v, t, buf, sd.p.st32);
  Best2F b;
  b.init();
#pragma unroll
  for (int u = 0; u < P; ++u) {
    const float2 x = v[fft_out_slot<float, LOGN>(u)];
    b.push_ascending(norm2<float>(x), t + TPF * u);
  }
  group_reduce<TPF>(b, red);
  if (t == 0 && active) {
    const float w2 = sd.p.wsq32[s];  // 1 - r_s^2 on this path
    Top2F o;
    o.v1 = b.v1 * w2;
    o.v2 = b.v2 * w2;
    o.j1 = b.j1;
    o.j2 = b.j2;
    reinterpret_cast<Top2F*>(sd.top2)[s] = o;
    if (o.v1 >= 0.0f && o.v1 <= 3.402823466e38f) atomicMax(&sd.ctl->vmax_bits, __float_as_uint(o.v1));
    __threadfence();  // read by the last CTA
  }
  if (!arrive_last(&sd.ctl->cnt_grid, gridDim.x, &s_last)) return;
  __shared__ SelectScratch scr;
  select_candidates_f32<THREADS>(sd, sd.ctl->k, 1, scr);
}

// w_m G(z_m) / (1 - a conj(z_m)) in FP64.
__device__ __forceinline__ double2 nu_term(double2 g, double w, double2 z, double ar, double ai) {
  // d = 1 - a conj(z)
  const double dr = 1.0 - fma(ar, z.x, ai * z.y);
  const double di = -fma(ai, z.x, -ar * z.y);
  const double inv = w / fma(dr, dr, di * di);
  // w g conj(d) / |d|^2
  return make_double2(fma(g.x, dr, g.y * di) * inv, fma(g.y, dr, -g.x * di) * inv);
}

// The FP64 guard: every candidate's weighted rectangle rule, split over CTAs
// as k_guard splits it; the last CTA picks the largest |c|^2 (ties: lowest
// flat index s N + j).
__global__ void __launch_bounds__(FP64_THREADS)
k_guard_nu(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  __shared__ double red[2 * (FP64_THREADS / 32)];
  __shared__ double s_re[MAX_CAP], s_im[MAX_CAP];
  __shared__ int s_last;
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[blockIdx.y]];
  SlotCtl* ctl = sd.ctl;
  pdl_wait();
  if (ld_done(ctl)) return;
  const int N = sd.p.N, n = sd.p.nN;
  const int Pg = chunks_of(n);
  const int c0 = blockIdx.x / Pg, p = blockIdx.x % Pg;
  const int n_cand = ctl->n_cand;
  const int m = p * FP64_CHUNK + threadIdx.x;
  double2 g = make_double2(0.0, 0.0), z = make_double2(1.0, 0.0);
  double w = 0.0;
  if (m < n && c0 < n_cand) {
    g = sd.G[m];
    z = __ldg(&sd.p.nz64[m]);
    w = __ldg(&sd.p.nw64[m]);
  }
  for (int c = c0; c < n_cand; c += GUARD_PAR) {
    const int2 cj = sd.cand[c];
    const double r = sd.p.radii[cj.x];
    const double2 wj = __ldg(&sd.p.tw64[cj.y]);
    double2 term = make_double2(0.0, 0.0);
    if (m < n) term = nu_term(g, w, z, r * wj.x, r * wj.y);
    const double2 tot = sum_fp64_group(term.x, term.y, red);
    if (threadIdx.x == 0) sd.gpart[c * Pg + p] = tot;
  }
  if (!arrive_last(&ctl->cnt_guard, gridDim.x, &s_last)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < n_cand; c += FP64_THREADS / 32) {
    double x = 0.0, y = 0.0;
    for (int q = lane; q < Pg; q += 32) {
      const double2 v = __ldcg(&sd.gpart[c * Pg + q]);
      x += v.x;
      y += v.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, off);
      y += __shfl_xor_sync(0xffffffffu, y, off);
    }
    if (lane == 0) {
      const double sc = sd.p.sq64[sd.cand[c].x];
      s_re[c] = sc * x;
      s_im[c] = sc * y;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int k = ctl->k;
  StepRec& rec = sd.rec[k];
  int bs = -1, bj = -1;
  double bv = -1.0, bre = 0.0, bim = 0.0;
  for (int c = 0; c < n_cand; ++c) {
    const int2 cj = sd.cand[c];
    const double v = s_re[c] * s_re[c] + s_im[c] * s_im[c];
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
  const double2 wj = sd.p.tw64[bj];
  rec.s = bs;
  rec.j = bj;
  rec.n_cand = n_cand;
  rec.a_re = rr * wj.x;
  rec.a_im = rr * wj.y;
  rec.c_re = bre;
  rec.c_im = bim;
  rec.obj = bv;
}

// The Blaschke update of Sec. 2 at the samples, with c' = c sqrt(1 - |a|^2):
//   G_{k+1}(z) = (G_k(z) (1 - conj(a) z) - c') / (z - a),
// the weighted energy sum_m w_m |G_{k+1}(z_m)|^2 (fixed-order sums as in
// k_update), delta, the stop rule, and w_m G_{k+1}(z_m) in FP32 for the next
// non-uniform DFT.  INIT: energy and FP32 copy of the starting remainder.
template <bool INIT>
__global__ void __launch_bounds__(FP64_THREADS)
k_update_nu(const SlotDev* __restrict__ slots, const int* __restrict__ ids) {
  __shared__ double red[2 * (FP64_THREADS / 32)];
  __shared__ int s_last;
  pdl_launch_dependents();
  const SlotDev& sd = slots[ids[blockIdx.y]];
  SlotCtl* ctl = sd.ctl;
  pdl_wait();
  if (ld_done(ctl)) return;
  const int n = sd.p.nN;
  const int Pu = chunks_of(n);
  const int p = blockIdx.x;
  const int m = p * FP64_CHUNK + threadIdx.x;
  const int k = ctl->k;
  double e = 0.0;
  if (m < n) {
    double2 g = sd.G[m];
    const double w = __ldg(&sd.p.nw64[m]);
    if constexpr (!INIT) {
      const StepRec& rec = sd.rec[k];
      const double na = sd.p.sq64[rec.s];
      const double cr = rec.c_re * na, ci = rec.c_im * na;
      const double ar = rec.a_re, ai = rec.a_im;
      const double2 z = __ldg(&sd.p.nz64[m]);
      // u = 1 - conj(a) z, x = g u - c'
      const double ur = 1.0 - fma(ar, z.x, ai * z.y);
      const double ui = -fma(ar, z.y, -ai * z.x);
      const double xr = fma(g.x, ur, fma(-g.y, ui, -cr));
      const double xi = fma(g.x, ui, fma(g.y, ur, -ci));
      // x / (z - a) = x conj(d) / |d|^2
      const double dr = z.x - ar, di = z.y - ai;
      const double inv = 1.0 / fma(dr, dr, di * di);
      g = make_double2(fma(xr, dr, xi * di) * inv, fma(xi, dr, -xr * di) * inv);
      sd.G[m] = g;
    }
    e = w * fma(g.x, g.x, g.y * g.y);
    sd.g32[m] = make_float2(d2f_rn(w * g.x), d2f_rn(w * g.y));  // integer-pipe conversion
  }
  const double es = sum_fp64_group1(e, red);
  if (threadIdx.x == 0) sd.epart[p] = es;
  if (!arrive_last(&ctl->cnt_update, gridDim.x, &s_last)) return;
  if (threadIdx.x >= 32) return;
  double E = 0.0;
  for (int q = threadIdx.x; q < Pu; q += 32) E += __ldcg(&sd.epart[q]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) E += __shfl_xor_sync(0xffffffffu, E, off);
  if (threadIdx.x != 0) return;
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

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_nu(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int LOGN>
cudaError_t grid_nu_launch(const SlotDev* slots, const int* ids, int M, cudaStream_t st) {
  using C = NuCfg<LOGN>;
  const dim3 grid((M + C::FPC - 1) / C::FPC, 1);
  return launch_pdl_nu(k_grid_nu<LOGN>, grid, dim3(C::THREADS), C::SMEM, st, slots, ids);
}

template <int LOGN>
cudaError_t grid_nu_attr() {
  return cudaFuncSetAttribute(k_grid_nu<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NuCfg<LOGN>::SMEM);
}

}  // namespace

cudaError_t launch_nudft(const SlotDev* slots, const int* ids, int Lc, cudaStream_t st) {
  const dim3 grid((Lc + NUDFT_L - 1) / NUDFT_L);
  return launch_pdl_nu(k_nudft, grid, dim3(NUDFT_THREADS), 0, st, slots, ids);
}

cudaError_t launch_grid_nu(const SlotDev* slots, const int* ids, int logN, int M, cudaStream_t st) {
  switch (logN) {
#define X(L) case L: return grid_nu_launch<L>(slots, ids, M, st);
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_guard_nu(const SlotDev* slots, const int* ids, int nN, int cap, cudaStream_t st) {
  const dim3 grid((cap < GUARD_PAR ? cap : GUARD_PAR) * chunks_of(nN), 1);
  return launch_pdl_nu(k_guard_nu, grid, dim3(FP64_THREADS), 0, st, slots, ids);
}

cudaError_t launch_update_nu(const SlotDev* slots, const int* ids, int nN, bool init, cudaStream_t st) {
  const dim3 grid(chunks_of(nN), 1);
  if (init) return launch_pdl_nu(k_update_nu<true>, grid, dim3(FP64_THREADS), 0, st, slots, ids);
  return launch_pdl_nu(k_update_nu<false>, grid, dim3(FP64_THREADS), 0, st, slots, ids);
}

cudaError_t nu_configure() {
  cudaError_t e;
#define X(L) if ((e = grid_nu_attr<L>()) != cudaSuccess) return e;
  X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)
#undef X
  return cudaSuccess;
}

}  // namespace afd
