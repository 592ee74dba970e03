// Device helpers shared by the kernel translation units: best-pair
// reductions, deterministic block sums, last-CTA detection, programmatic
// dependent launch, and the selection of Step 2 (Sec. 3.2) run by the last CTA
// of a signal's grid launch.
#pragma once
#include <climits>
#include <cstdint>
#include <type_traits>

#include "afd_internal.h"

namespace afd {


__device__ __forceinline__ bool better_f(float va, int ja, float vb, int jb) {
  return va > vb || (va == vb && ja < jb);
}
__device__ __forceinline__ bool better_d(double va, int ja, double vb, int jb) {
  return va > vb || (va == vb && ja < jb);
}

// FP64 -> FP32 rounded to nearest even, on the integer pipe.  A cast is an
// FP64-pipe instruction, as slow as a multiply on this chip.  Results below
// 2^-126 in magnitude flush to zero; overflow gives infinity, NaN stays NaN.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int ex = (int)((hi >> 20) & 0x7ffu);
  if (ex == 0x7ff) return __int_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
  const int e = ex - 1023 + 127;
  if (e <= 0) return __int_as_float(sign);
  if (e >= 255) return __int_as_float(sign | 0x7f800000u);
  // keep 23 of the 52 fraction bits; the 29 dropped ones decide the rounding
  unsigned r = ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ++r;  // a carry into the exponent is right
  return __int_as_float(sign | r);
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Best2F {
  float v1, v2;
  int j1, j2;
  __device__ __forceinline__ void init() { v1 = v2 = -1.0f; j1 = j2 = INT_MAX; }
  __device__ __forceinline__ void insert(float v, int j) {
    if (better_f(v, j, v1, j1)) { v2 = v1; j2 = j1; v1 = v; j1 = j; }
    else if (better_f(v, j, v2, j2)) { v2 = v; j2 = j; }
  }
  // For values offered in increasing index order: the index exceeds every
  // index held, so a tie keeps the held (lower) one and plain comparisons do.
  __device__ __forceinline__ void push_ascending(float v, int j) {
    const bool p1 = v > v1, p2 = v > v2;
    v2 = p1 ? v1 : (p2 ? v : v2);
    j2 = p1 ? j1 : (p2 ? j : j2);
    v1 = p1 ? v : v1;
    j1 = p1 ? j : j1;
  }
  // both pairs ordered (first better than second); selects, no branches
  __device__ __forceinline__ void merge(const Best2F& o) {
    const bool a = better_f(o.v1, o.j1, v1, j1);
    const bool b1 = better_f(v1, j1, o.v2, o.j2);
    const bool b2 = better_f(o.v1, o.j1, v2, j2);
    const float nv2 = a ? (b1 ? v1 : o.v2) : (b2 ? o.v1 : v2);
    const int nj2 = a ? (b1 ? j1 : o.j2) : (b2 ? o.j1 : j2);
    v1 = a ? o.v1 : v1;
    j1 = a ? o.j1 : j1;
    v2 = nv2;
    j2 = nj2;
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
  __device__ __forceinline__ void push_ascending(double vv, int jj, double2 ff) {
    const bool p = vv > v;
    v = p ? vv : v;
    j = p ? jj : j;
    f = p ? ff : f;
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

// The best two (value, index) pairs of a whole warp's Best2F, in every lane,
// by four warp reductions instead of a shuffle tree: the best is the largest
// v1 (lowest index on ties); the second is the best of the owner lane's
// (v2, j2) and every other lane's (v1, j1), since a lane's second pair never
// beats its first.  The values are >= -1 and never NaN (push_ascending and
// merge keep NaN out), so their order is the float order; indices are
// distinct.  Bitwise the result of the shuffle-tree merge.
__device__ __forceinline__ void warp_top2(Best2F& b) {
  float v1, v2;
  unsigned j1, j2;
  asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(v1) : "f"(b.v1));
  asm volatile("redux.sync.min.u32 %0, %1, 0xffffffff;" : "=r"(j1) : "r"(b.v1 == v1 ? (unsigned)b.j1 : 0xffffffffu));
  const bool own = (unsigned)b.j1 == j1;
  const float cv = own ? b.v2 : b.v1;
  const unsigned cj = (unsigned)(own ? b.j2 : b.j1);
  asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(v2) : "f"(cv));
  asm volatile("redux.sync.min.u32 %0, %1, 0xffffffff;" : "=r"(j2) : "r"(cv == v2 ? cj : 0xffffffffu));
  b.v1 = v1;
  b.j1 = (int)j1;
  b.v2 = v2;
  b.j2 = (int)j2;
}

// Reduce B over each group of TPF consecutive threads; the group's thread
// t == 0 ends with the result.  All threads of the CTA must call it.
// FRESH: red was last read before a CTA barrier the caller has passed since,
// so the barrier that protects its reuse can be skipped.
template <int TPF, class B, bool FRESH = false>
__device__ __forceinline__ void group_reduce(B& b, B* red) {
  constexpr int W = TPF < 32 ? TPF : 32;
  constexpr bool REDUX = std::is_same<B, Best2F>::value && TPF >= 32;
  if constexpr (REDUX) {
    warp_top2(b);
  } else {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) b.merge(b.shfl(off));
  }
  if constexpr (TPF > 32) {
    // the group's warp results, merged by a shuffle tree in its first warp
    // (the best pair of a set of distinct indices does not depend on the
    // order of the merges)
    constexpr int WPG = TPF / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (!FRESH) __syncthreads();
    if (lane == 0) red[warp] = b;
    __syncthreads();
    if ((warp % WPG) == 0) {
      B o;
      if (lane < WPG) o = red[warp + lane];
      else o.init();
      if constexpr (REDUX) {
        warp_top2(o);
      } else {
#pragma unroll
        for (int off = WPG / 2; off > 0; off >>= 1) o.merge(o.shfl(off));
      }
      if (lane == 0) b = o;
    }
  }
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

// A set of threads that works and synchronises as one unit: the whole CTA
// (barrier 0), or a part of it on its own named barrier (bar > 0, count
// threads).  tid: the thread's index within the set.
struct ThreadSet {
  int bar, count, tid;
  __device__ __forceinline__ void sync() const {
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(count) : "memory");
  }
};
__device__ __forceinline__ ThreadSet cta_set() { return ThreadSet{0, (int)blockDim.x, (int)threadIdx.x}; }

// Last-work-item detection: returns true in every thread of the set that is
// the last of `target` items to arrive on *counter, and resets the counter.
// Every write the last item reads must come from thread 0 of its set or be
// followed by a __threadfence() in the thread that made it.
__device__ __forceinline__ bool arrive_last_set(unsigned* counter, unsigned target, int* s_flag, const ThreadSet& ts) {
  ts.sync();
  if (ts.tid == 0) {
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    *s_flag = (prev == target - 1u);
    if (*s_flag) *counter = 0u;
  }
  ts.sync();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}
// The same for the whole CTA (one CTA per work item).
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned target, int* s_flag) {
  return arrive_last_set(counter, target, s_flag, cta_set());
}

constexpr long kBarrierLimit = 1L << 22;  // polls before a grid barrier gives up (about a second)

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch (all CTAs are co-resident).  The
// arrival counter *bar only grows during a launch (the host zeroes it
// before), so barrier number e of the launch is passed once it reaches
// nblocks * (e + 1): one reduction per CTA and a poll, no reset.  Thread 0
// arrives with a release reduction (after the CTA barrier, so it publishes
// the CTA's writes) and polls with acquire loads, so the others' writes are
// visible once the count is reached.  Bounded: a CTA that polls
// kBarrierLimit times sets bit 2 (value 4) of *err, and every CTA that sees
// the bit leaves.  False in every thread when the kernel must stop.
__device__ __forceinline__ bool grid_barrier_at(unsigned* bar, int* err, unsigned target, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    for (long it = 1; ld_acquire_gpu(bar) < target; ++it) {
      if (it > kBarrierLimit) {
        atomicOr(err, 4);
        ok = 0;
        break;
      }
      if ((it & 255) == 0 && (*((volatile int*)err) & 4)) {  // another CTA gave up
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    if (*((volatile int*)err) & 4) ok = 0;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Four doubles read with one 256-bit load through L2 (32-byte aligned).
struct double4v {
  double x, y, z, w;
};
__device__ __forceinline__ double4v ld_cg_v4(const double* p) {
  double4v r;
  asm volatile("ld.global.cg.v4.f64 {%0, %1, %2, %3}, [%4];"
               : "=d"(r.x), "=d"(r.y), "=d"(r.z), "=d"(r.w)
               : "l"(p)
               : "memory");
  return r;
}

__device__ __forceinline__ int ld_done(const SlotCtl* c) { return *((volatile const int*)&c->done); }

// Programmatic dependent launch: the step kernels are launched so that the
// next kernel in the stream may be scheduled while this one runs.  Each kernel
// lets its dependents launch at entry and waits for its own predecessor to
// complete (with its memory visible) before reading anything it produced.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Candidates of the FP32 path: every grid point whose FP32 objective is at
// least thr, ordered best first (value, then lowest flat index s N + j); the
// first cap of them go to out[].  Reads the best pairs top[0 .. M sub), sub
// entries per radius.  Every thread of the CTA must call it; every thread gets
// n (candidates kept) and count (points at or above thr).  Deterministic: the
// same inputs give the same list in any CTA.
// The candidate list's shared-memory scratch (8 KB): the caller's own, or a
// buffer of its that is free by then (a grid kernel's transform buffers).
struct SelectScratch {
  static constexpr int LIST = 1024;
  float v[LIST];
  int f[LIST];
};
template <int THREADS>
__device__ void select_core(const Top2F* top, int M, int N, int sub, float thr, int cap, int2* out, int* n_out,
                            int* count_out, SelectScratch& scr) {
  constexpr int LIST = SelectScratch::LIST;
  float* s_v = scr.v;
  int* s_f = scr.f;
  __shared__ int s_count;
  __shared__ float sv[32];
  __shared__ int sf[32];
  // (the buffers above are this function's own: every read of them comes
  // before the CTA barrier that ends the previous call)
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < M * sub; r += THREADS) {
    const int s = r / sub;
    const int4 raw = __ldcg(reinterpret_cast<const int4*>(top) + r);  // v1, v2, j1, j2
    const float v1 = __int_as_float(raw.x), v2 = __int_as_float(raw.y);
    if (v1 >= thr && raw.z != INT_MAX) {
      const int i = atomicAdd(&s_count, 1);
      if (i < LIST) { s_v[i] = v1; s_f[i] = s * N + raw.z; }
    }
    if (v2 >= thr && raw.w != INT_MAX) {
      const int i = atomicAdd(&s_count, 1);
      if (i < LIST) { s_v[i] = v2; s_f[i] = s * N + raw.w; }
    }
  }
  __syncthreads();
  const int count = s_count;
  int n;
  if (count <= LIST) {
    // rank of each entry = number of better entries; ranks are distinct
    for (int i = threadIdx.x; i < count; i += THREADS) {
      const float v = s_v[i];
      const int f = s_f[i];
      int rank = 0;
      for (int q = 0; q < count; ++q) rank += better_f(s_v[q], s_f[q], v, f) ? 1 : 0;
      if (rank < cap) out[rank] = make_int2(f / N, f % N);
    }
    n = min(count, cap);
  } else {
    // a plateau wider than the list (degenerate input): pick the best cap one
    // at a time, each strictly worse than the previous pick
    float last_v = __int_as_float(0x7f800000);
    int last_f = -1;
    for (n = 0; n < cap; ++n) {
      float bv = -1.0f;
      int bf = INT_MAX;
      for (int e = threadIdx.x; e < 2 * M * sub; e += THREADS) {
        const int r = e >> 1, s = r / sub;
        const float v = (e & 1) ? __ldcg(&top[r].v2) : __ldcg(&top[r].v1);
        const int j = (e & 1) ? __ldcg(&top[r].j2) : __ldcg(&top[r].j1);
        if (j == INT_MAX || !(v >= thr)) continue;
        const int f = s * N + j;
        if (better_f(last_v, last_f, v, f) && better_f(v, f, bv, bf)) { bv = v; bf = f; }
      }
      block_best_f<THREADS>(bv, bf, sv, sf);
      if (bf == INT_MAX) break;
      if (threadIdx.x == 0) out[n] = make_int2(bf / N, bf % N);
      last_v = bv;
      last_f = bf;
    }
  }
  __syncthreads();
  *n_out = n;
  *count_out = count;
}

// FP32 selection in the last CTA of a signal's grid launch: every grid point
// whose FP32 objective is within the relative window tau of the step's largest
// one (known from the atomicMax each CTA made) becomes a candidate for the
// FP64 guard, at most cap of them, best first.
template <int THREADS>
__device__ void select_candidates_f32(const SlotDev& sd, int k, int sub, SelectScratch& scr) {
  SlotCtl* ctl = sd.ctl;
  StepRec& rec = sd.rec[k];
  const float vmax = __uint_as_float(__ldcg(&ctl->vmax_bits));
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->vmax_bits = 0u;  // ready for the next step
    rec.obj32 = vmax;
    rec.flags = 0;
  }
  if (sd.force_a1_zero && k == 0) {
    if (threadIdx.x == 0) {
      sd.cand[0] = make_int2(0, 0);
      ctl->n_cand = 1;
    }
    return;
  }
  const float thr = vmax - vmax * (float)sd.tau;
  int n, count;
  select_core<THREADS>(reinterpret_cast<const Top2F*>(sd.top2), sd.p.M, sd.p.N, sub, thr, sd.cap, sd.cand, &n,
                       &count, scr);
  if (threadIdx.x == 0) {
    ctl->n_cand = n;
    if (count > sd.cap) rec.flags = 1;
  }
}

// ---------------------------------------------------- FP64 guard and update --

// One term of the guard's rectangle rule for the candidate (s, j) at sample m:
// G(z_m) K_s[(j - m) mod N], K_s[d] = 1 / (1 - r_s w^d).
__device__ __forceinline__ void guard_term(const SlotDev& sd, int s, int j, int m, double2 g, double& ar,
                                           double& ai) {
  const int N = sd.p.N;
  const double2 k = __ldg(&sd.p.K64[(size_t)s * N + wrap_mod(j - m, N)]);
  ar = fma(g.x, k.x, -g.y * k.y);
  ai = fma(g.x, k.y, g.y * k.x);
}

// Fixed-order sum over the first FP64_THREADS threads (warps 0..3) of a
// thread set of (x, y): a shuffle tree inside each warp, then the warps in
// order.  Every thread of the set must call it; its thread 0 gets the total.
__device__ __forceinline__ double2 sum_fp64_set(double x, double y, double* red, const ThreadSet& ts) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, off);
    y += __shfl_xor_sync(0xffffffffu, y, off);
  }
  const int lane = ts.tid & 31, warp = ts.tid >> 5;
  ts.sync();
  if (lane == 0 && warp < FP64_THREADS / 32) {
    red[2 * warp] = x;
    red[2 * warp + 1] = y;
  }
  ts.sync();
  double tx = 0.0, ty = 0.0;
  if (ts.tid == 0) {
#pragma unroll
    for (int w = 0; w < FP64_THREADS / 32; ++w) {
      tx += red[2 * w];
      ty += red[2 * w + 1];
    }
  }
  return make_double2(tx, ty);
}
__device__ __forceinline__ double2 sum_fp64_group(double x, double y, double* red) {
  return sum_fp64_set(x, y, red, cta_set());
}

// The same for one component (the energy): the x half of sum_fp64_set,
// bitwise the same total.
__device__ __forceinline__ double sum_fp64_set1(double x, double* red, const ThreadSet& ts) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  const int lane = ts.tid & 31, warp = ts.tid >> 5;
  ts.sync();
  if (lane == 0 && warp < FP64_THREADS / 32) red[warp] = x;
  ts.sync();
  double tx = 0.0;
  if (ts.tid == 0) {
#pragma unroll
    for (int w = 0; w < FP64_THREADS / 32; ++w) tx += red[w];
  }
  return tx;
}
__device__ __forceinline__ double sum_fp64_group1(double x, double* red) { return sum_fp64_set1(x, red, cta_set()); }

// Reduced-remainder update of Sec. 2 at z_m for a = r_s w^j and
// c' = c sqrt(1 - r_s^2):  G_{k+1}(z_m) = (G_k(z_m) u - c') / (z_m - a) with
// u = 1 - conj(a) z_m = 1 - r_s w^d, d = (m - j) mod N.  Because
// z_m - a = z_m conj(u), dividing by it is multiplying by
// B = conj(z_m) conj(K_s[d]), so G_{k+1}(z_m) = (U - c') B with U = G_k(z_m) u.
// U and B depend on the selected point but not on its coefficient, so the
// persistent kernel forms them while the coefficient is still being summed.
// (Ten FP64 operations for U and B, six to apply: FP64 is the scarce pipe.)
struct UpdCoef {
  double2 U, B;
};
__device__ __forceinline__ UpdCoef update_coef(const SlotDev& sd, int m, int s, int j, double r, double2 g) {
  const int N = sd.p.N;
  const int d = wrap_mod(m - j, N);
  const double2 w = __ldg(&sd.p.tw64[d]);
  const double2 z = __ldg(&sd.p.tw64[m]);
  const double2 kd = __ldg(&sd.p.K64[(size_t)s * N + d]);
  const double ur = fma(-r, w.x, 1.0), ui = -r * w.y;
  // B = conj(K z)
  const double br = fma(kd.x, z.x, -kd.y * z.y);
  const double bi = -fma(kd.x, z.y, kd.y * z.x);
  UpdCoef o;
  o.U = make_double2(fma(g.x, ur, -g.y * ui), fma(g.x, ui, g.y * ur));
  o.B = make_double2(br, bi);
  return o;
}
// The two halves of update_coef on their own (bitwise the same values), for
// forming them on two warps: U = G u and B = conj(K z).
__device__ __forceinline__ double2 update_u(const SlotDev& sd, int m, int j, double r, double2 g) {
  const double2 w = __ldg(&sd.p.tw64[wrap_mod(m - j, sd.p.N)]);
  const double ur = fma(-r, w.x, 1.0), ui = -r * w.y;
  return make_double2(fma(g.x, ur, -g.y * ui), fma(g.x, ui, g.y * ur));
}
__device__ __forceinline__ double2 update_b(const SlotDev& sd, int m, int s, int j) {
  const int N = sd.p.N;
  const double2 z = __ldg(&sd.p.tw64[m]);
  const double2 kd = __ldg(&sd.p.K64[(size_t)s * N + wrap_mod(m - j, N)]);
  return make_double2(fma(kd.x, z.x, -kd.y * z.y), -fma(kd.x, z.y, kd.y * z.x));
}
__device__ __forceinline__ double2 update_apply(const UpdCoef& q, double cr, double ci) {
  const double xr = q.U.x - cr, xi = q.U.y - ci;
  return make_double2(fma(xr, q.B.x, -xi * q.B.y), fma(xr, q.B.y, xi * q.B.x));
}
__device__ __forceinline__ double2 update_point(const SlotDev& sd, int m, int s, int j, double r, double cr,
                                                double ci, double2 g) {
  return update_apply(update_coef(sd, m, s, j, r, g), cr, ci);
}

// FP64 selection: global best of the per-radius maxima (sub entries per
// radius: one per sub-transform of a split size); writes the step record.
template <int THREADS>
__device__ void select_best_f64(const SlotDev& sd, int k, Best1D* red, int sub = 1) {
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
    for (int e = threadIdx.x; e < M * sub; e += THREADS) {
      const int j = __ldcg(&top[e].j1);
      if (j == INT_MAX) continue;
      double2 f;
      f.x = __ldcg(&top[e].f1.x);
      f.y = __ldcg(&top[e].f1.y);
      b.insert(__ldcg(&top[e].v1), (e / sub) * N + j, f);
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
    r.obj = (r.c_re * r.c_re + r.c_im * r.c_im) * obj_rho64(sd, s);
    r.obj32 = b.v;
  }
}


}  // namespace afd
