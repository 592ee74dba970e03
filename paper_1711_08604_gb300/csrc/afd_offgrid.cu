// Off-grid refinement of the selected point (optional, sm_103a).
//
// The paper selects a_k on the polar grid of Sec. 3.2.  With
// afd_plan_opts.offgrid_iters > 0 a plan refines each step's grid winner a0
// over the open disc before the coefficient and the update, maximising the
// same discrete objective off the grid:
//   f(a) = |<G_k, e_a>~|^2 = (1 - |a|^2) |S(a)|^2 / N^2,
//   S(a) = sum_m G_k(z_m) / (1 - a conj(z_m))          (Eq. (formula1)),
// by damped Newton steps on h = log f in the real coordinates (x, y) of a.
// S is holomorphic in a, so 2 Re log S is harmonic and, with L1 = S'/S and
// L2 = S''/S - L1^2, rho = 1 - |a|^2:
//   grad h = (2 Re L1 - 2x/rho, -2 Im L1 - 2y/rho),
//   h_xx = 2 Re L2 - 2/rho - 4x^2/rho^2,   h_xy = -2 Im L2 - 4xy/rho^2,
//   h_yy = -2 Re L2 - 2/rho - 4y^2/rho^2,
//   S'(a) = sum G conj(z) / (1 - a conj(z))^2,  S''(a) = 2 sum G conj(z)^2 / (1 - a conj(z))^3.
// An iteration stops the refinement unless the Hessian is negative definite;
// a Newton step shorter than 1e-6 is taken as it is (near the maximum f no
// longer resolves the gain, and the convergence is quadratic); a longer one,
// shortened to at most half the distance to the circle, is tried and then
// halved up to three times, and taken at the first try that increases f
// (none: stop).  A step shorter than 1e-13 ends it.  The coefficient is
// <G_k, e_a>~ = sqrt(1 - |a|^2) S(a) / N at the final a.
//
// k_refine: a cooperative launch of up to RF_MAX_CTAS CTAs per signal; every
// pass over the samples sums S, S', S'' at one point (per-CTA partials, a
// bounded grid barrier, the partials added in a fixed order by every CTA),
// and every CTA takes the same decisions.  It writes the refined a, the
// coefficient and |c|^2 into the step record (flag bit 3) and keeps the grid
// indices (s, j) of the starting point.
// k_update_offgrid: the remainder update of Sec. 2 at a point off the grid,
//   G_{k+1}(z_m) = (G_k(z_m) u - c') / (z_m - a),  u = 1 - conj(a) z_m,  c' = c sqrt(1 - |a|^2),
// with z_m - a = z_m conj(u) (|z_m| = 1), so dividing is multiplying by
// conj(z_m) u / |u|^2; energy, delta and the stop rule as the grid update.
#include <cstdint>

#include "../../include/afd.h"
#include "afd_device.cuh"
#include "afd_internal.h"

namespace afd {

namespace {

constexpr int RF_THREADS = 128;
constexpr int RF_WARPS = RF_THREADS / 32;

struct C2 {
  double x, y;
};
__device__ __forceinline__ C2 cm(C2 a, C2 b) { return C2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
// a / b
__device__ __forceinline__ C2 cdiv(C2 a, C2 b) {
  const double q = 1.0 / (b.x * b.x + b.y * b.y);
  return C2{(a.x * b.x + a.y * b.y) * q, (a.y * b.x - a.x * b.y) * q};
}

__device__ __forceinline__ double rf_f(C2 a, C2 S) { return (1.0 - (a.x * a.x + a.y * a.y)) * (S.x * S.x + S.y * S.y); }

// The refinement of one signal by a cooperative launch of C <= RF_MAX_CTAS
// CTAs: CTA b sums the samples [b N / C, (b + 1) N / C) of every pass (each
// thread its samples in order, a fixed shuffle tree, the warps in order),
// posts its six partials, and after a bounded grid barrier every CTA adds the
// C partials in the same order (lane q: partials q, q + 32, then a fixed
// tree), so every CTA takes the same decisions.  The partials alternate
// between two buffers by pass parity.  The barrier counter continues across
// launches: ctl->bar_gen holds the barriers passed so far.
__global__ void __launch_bounds__(RF_THREADS) k_refine(const SlotDev* __restrict__ slots, const int* __restrict__ ids,
                                                       int iters) {
  __shared__ double red[6][RF_WARPS];
  __shared__ double s_tot[6];
  __shared__ double s_try[2];
  __shared__ int s_go, s_ok;
  const SlotDev& sd = slots[ids[0]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const int k = ctl->k;
  StepRec& rec = sd.rec[k];
  if (sd.force_a1_zero && k == 0) return;  // a_1 = 0 is imposed, not selected
  const int N = sd.p.N, C = (int)gridDim.x, b = (int)blockIdx.x;
  const int lo = (int)((long long)b * N / C), hi = (int)((long long)(b + 1) * N / C);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned epoch = ctl->bar_gen;  // the same in every CTA: written by the last launch
  int pass = 0;
  bool ok = true;
  // S, S', S'' at a: every thread gets them (false on a barrier timeout)
  auto sums = [&](C2 a, C2* S0, C2* S1, C2* S2) -> bool {
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int m = lo + (int)threadIdx.x; m < hi; m += RF_THREADS) {
      const double2 zz = __ldg(&sd.p.tw64[m]);
      const double2 gg = sd.G[m];
      const C2 zb{zz.x, -zz.y};
      const C2 d = C2{1.0 - (a.x * zb.x - a.y * zb.y), -(a.x * zb.y + a.y * zb.x)};
      const double q = 1.0 / (d.x * d.x + d.y * d.y);
      const C2 v{d.x * q, -d.y * q};  // 1 / (1 - a conj(z))
      const C2 t = cm(C2{gg.x, gg.y}, v);
      const C2 w = cm(zb, v);
      const C2 tw = cm(t, w);
      const C2 tww = cm(tw, w);
      acc[0] += t.x;
      acc[1] += t.y;
      acc[2] += tw.x;
      acc[3] += tw.y;
      acc[4] += 2.0 * tww.x;
      acc[5] += 2.0 * tww.y;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double x = acc[i];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if (lane == 0) red[i][warp] = x;
    }
    __syncthreads();
    double* part = sd.rfpart + (size_t)(pass & 1) * RF_MAX_CTAS * 6;
    if (threadIdx.x < 6) {
      double x = 0.0;
      for (int w = 0; w < RF_WARPS; ++w) x += red[threadIdx.x][w];
      part[b * 6 + threadIdx.x] = x;
    }
    ++pass;
    if (!grid_barrier_at(sd.bar, &ctl->err, (unsigned)C * ++epoch, &s_ok)) return false;
    // every CTA: the C partials in a fixed order (warp w: components w, w + 4)
    for (int i = warp; i < 6; i += RF_WARPS) {
      double x = 0.0;
      for (int q = lane; q < C; q += 32) x += __ldcg(&part[q * 6 + i]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if (lane == 0) s_tot[i] = x;
    }
    __syncthreads();
    *S0 = C2{s_tot[0], s_tot[1]};
    *S1 = C2{s_tot[2], s_tot[3]};
    *S2 = C2{s_tot[4], s_tot[5]};
    __syncthreads();  // red and s_tot are reused by the next pass
    return true;
  };
  C2 a{rec.a_re, rec.a_im};
  C2 S, S1, S2;
  ok = sums(a, &S, &S1, &S2);
  double f = rf_f(a, S);
  for (int it = 0; ok && it < iters; ++it) {
    // thread 0 of every CTA decides (the same in every CTA); its CTA follows
    double dx = 0.0, dy = 0.0;
    int mode = 0;  // 0 stop, 1 take the small step, 2 damped trials, 3 take it and stop
    if (threadIdx.x == 0 && (S.x != 0.0 || S.y != 0.0)) {
      const C2 L1 = cdiv(S1, S);
      const C2 q = cdiv(S2, S);
      const C2 L2 = C2{q.x - (L1.x * L1.x - L1.y * L1.y), q.y - 2.0 * L1.x * L1.y};
      const double x = a.x, y = a.y;
      const double rho = 1.0 - (x * x + y * y);
      const double gx = 2.0 * L1.x - 2.0 * x / rho;
      const double gy = -2.0 * L1.y - 2.0 * y / rho;
      const double hxx = 2.0 * L2.x - 2.0 / rho - 4.0 * x * x / (rho * rho);
      const double hxy = -2.0 * L2.y - 4.0 * x * y / (rho * rho);
      const double hyy = -2.0 * L2.x - 2.0 / rho - 4.0 * y * y / (rho * rho);
      const double det = hxx * hyy - hxy * hxy;
      if (det > 0.0 && hxx < 0.0) {
        dx = -(hyy * gx - hxy * gy) / det;
        dy = -(hxx * gy - hxy * gx) / det;
        const double lim = 0.5 * (1.0 - sqrt(x * x + y * y));
        const double n = sqrt(dx * dx + dy * dy);
        if (n < 1e-6 && n < lim) {
          mode = n < 1e-13 ? 3 : 1;
        } else {
          if (n > lim) {
            dx *= lim / n;
            dy *= lim / n;
          }
          mode = 2;
        }
      }
      s_try[0] = dx;
      s_try[1] = dy;
      s_go = mode;
    }
    __syncthreads();
    mode = s_go;
    dx = s_try[0];
    dy = s_try[1];
    __syncthreads();  // s_go and s_try are rewritten below
    if (mode == 0) break;
    if (mode == 1 || mode == 3) {
      a = C2{a.x + dx, a.y + dy};
      ok = sums(a, &S, &S1, &S2);
      f = rf_f(a, S);
      if (mode == 3) break;
      continue;
    }
    bool taken = false;
    for (int h = 0; ok && h < 4 && !taken; ++h) {
      const C2 an{a.x + dx, a.y + dy};
      C2 T, T1, T2;
      ok = sums(an, &T, &T1, &T2);
      const double fn = rf_f(an, T);  // the same value in every thread of every CTA
      if (fn > f) {
        a = an;
        S = T;
        S1 = T1;
        S2 = T2;
        f = fn;
        taken = true;
      } else {
        dx *= 0.5;
        dy *= 0.5;
      }
    }
    if (!taken) break;
    if (sqrt(dx * dx + dy * dy) < 1e-13) break;
  }
  if (!ok) {
    if (threadIdx.x == 0) ctl->done = 1;  // the barrier gave up: error bit 2 is set
    return;
  }
  if (b == 0 && threadIdx.x == 0) {
    // every CTA has passed the last barrier, so every CTA has read bar_gen
    ctl->bar_gen = epoch;
    const double na = sqrt(1.0 - (a.x * a.x + a.y * a.y)) / (double)N;
    const double cr = S.x * na, ci = S.y * na;
    rec.a_re = a.x;
    rec.a_im = a.y;
    rec.c_re = cr;
    rec.c_im = ci;
    rec.obj = cr * cr + ci * ci;
    rec.flags |= 8;
  }
}

// The remainder update at a point off the grid (rec.a_re, rec.a_im), one
// 128-sample chunk per CTA, with update_body's energy partials, last-CTA
// totals, delta and stop rule.
__global__ void __launch_bounds__(FP64_THREADS) k_update_offgrid(const SlotDev* __restrict__ slots,
                                                                 const int* __restrict__ ids) {
  __shared__ double red[FP64_THREADS / 32];
  __shared__ double s_cp[4];
  __shared__ int s_last;
  pdl_launch_dependents();
  pdl_wait();
  const SlotDev& sd = slots[ids[blockIdx.y]];
  SlotCtl* ctl = sd.ctl;
  if (ld_done(ctl)) return;
  const ThreadSet ts = cta_set();
  const int N = sd.p.N;
  const int Pu = chunks_of(N);
  const int p = blockIdx.x;
  const int m = p * FP64_CHUNK + threadIdx.x;
  const int k = ctl->k;
  if (threadIdx.x == 0) {
    const StepRec& rec = sd.rec[k];
    const double na = sqrt(1.0 - (rec.a_re * rec.a_re + rec.a_im * rec.a_im));
    s_cp[0] = rec.c_re * na;
    s_cp[1] = rec.c_im * na;
    s_cp[2] = rec.a_re;
    s_cp[3] = rec.a_im;
  }
  __syncthreads();
  double e = 0.0;
  if (m < N) {
    const double2 z = __ldg(&sd.p.tw64[m]);
    const double2 g = sd.G[m];
    const double ar = s_cp[2], ai = s_cp[3];
    // u = 1 - conj(a) z
    const double ur = 1.0 - (ar * z.x + ai * z.y), ui = -(ar * z.y - ai * z.x);
    const double xr = g.x * ur - g.y * ui - s_cp[0], xi = g.x * ui + g.y * ur - s_cp[1];  // G u - c'
    // conj(z) u / |u|^2
    const double q = 1.0 / (ur * ur + ui * ui);
    const double br = (z.x * ur + z.y * ui) * q, bi = (z.x * ui - z.y * ur) * q;
    const double2 gn = make_double2(xr * br - xi * bi, xr * bi + xi * br);
    sd.G[m] = gn;
    e = gn.x * gn.x + gn.y * gn.y;
    if (sd.prec) {
      const float inv_n = d2f_rn(sd.p.inv_n);
      sd.g32[m] = make_float2(d2f_rn(gn.x) * inv_n, d2f_rn(gn.y) * inv_n);
    }
  }
  const double es = sum_fp64_set1(e, red, ts);
  if (threadIdx.x == 0) sd.epart[p] = es;
  if (!arrive_last_set(&ctl->cnt_update, gridDim.x, &s_last, ts)) return;
  if (threadIdx.x >= 32) return;
  double E = 0.0;
  for (int q = threadIdx.x; q < Pu; q += 32) E += __ldcg(&sd.epart[q]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) E += __shfl_xor_sync(0xffffffffu, E, off);
  if (threadIdx.x != 0) return;
  E /= (double)N;
  StepRec& rec = sd.rec[k];
  const double delta = ctl->E1 > 0.0 ? E / ctl->E1 : 0.0;
  rec.energy = E;
  rec.delta = delta;
  ctl->k = k + 1;
  if (k + 1 >= sd.K_max || (sd.tol > 0.0 && delta <= sd.tol)) ctl->done = 1;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_og(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

cudaError_t launch_refine(const SlotDev* slots, const int* ids, int n, int N, int iters, cudaStream_t st) {
  if (n <= 0 || iters <= 0) return cudaSuccess;
  if (n != 1) return cudaErrorInvalidValue;  // plans: one signal
  // one CTA per 128 samples, at most RF_MAX_CTAS, all co-resident (cooperative)
  int C = chunks_of(N);
  if (C > RF_MAX_CTAS) C = RF_MAX_CTAS;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(RF_THREADS);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_refine, slots, ids, iters);
}

cudaError_t launch_update_offgrid(const SlotDev* slots, const int* ids, int n, int N, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  return launch_pdl_og(k_update_offgrid, dim3(chunks_of(N), n), dim3(FP64_THREADS), st, slots, ids);
}

}  // namespace afd
