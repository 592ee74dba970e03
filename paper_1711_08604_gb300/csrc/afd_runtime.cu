// Host runtime of the Core AFD library: plans, single-signal decomposition and
// batches of uneven N.  Implements the C ABI declared in include/afd.h.
//
// Device memory layout.  A plan owns the tables of one (N, radii) pair: the
// FP64 sample points / twiddles z_k = exp(2 pi i k / N) and their FP32
// rounding, the radial power tables r_s^q and r_s^(B h) (B = min(64, N)) in
// FP64 and FP32, and the per-radius scales.  Every signal in flight owns a
// slot: its FP64 remainder G_k, its spectrum, the per-radius best pairs, the
// guard candidates and partial sums, the step records and a control block.
// A batch allocates all slots in one pooled buffer, arrays of one kind laid
// out signal after signal, so a packed input is copied in with one memcpy.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/afd.h"
#include "afd_fft.cuh"
#include "afd_fft2.h"
#include "afd_host.h"
#include "afd_internal.h"

using namespace afd;

// ------------------------------------------------------------------ errors --

namespace afd {

namespace {
thread_local std::string g_last_error;
std::mutex g_cfg_mu;
bool g_configured[64] = {};
}  // namespace

afd_status set_error(afd_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

void set_last_error_text(const char* text) { g_last_error = text ? text : ""; }
void clear_last_error() { g_last_error.clear(); }
const char* last_error_text() { return g_last_error.c_str(); }

afd_status cuda_fail(cudaError_t e, const char* what, int line) {
  cudaGetLastError();  // clear a non-sticky error
  return set_error(e == cudaErrorMemoryAllocation ? AFD_ERR_NOMEM : AFD_ERR_CUDA,
                   "%s failed (line %d): %s", what, line, cudaGetErrorString(e));
}

afd_status ensure_configured(int dev) {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  if (dev < 0 || dev >= 64) return set_error(AFD_ERR_INVALID, "device ordinal %d out of range", dev);
  if (g_configured[dev]) return AFD_OK;
  CUDA_TRY(configure_kernels());
  g_configured[dev] = true;
  return AFD_OK;
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

afd_status check_opts(const afd_plan_opts& o) {
  if (o.precision != AFD_FP64_PLAIN && o.precision != AFD_FP32_GUARDED)
    return set_error(AFD_ERR_INVALID, "precision must be AFD_FP64_PLAIN or AFD_FP32_GUARDED");
  if (!(o.guard_tau >= 0.0 && o.guard_tau < 1.0))
    return set_error(AFD_ERR_INVALID, "guard_tau must lie in [0, 1)");
  if (o.guard_cap < 1 || o.guard_cap > MAX_CAP)
    return set_error(AFD_ERR_INVALID, "guard_cap must lie in 1..%d", MAX_CAP);
  if (o.grid_variant < -1 || o.grid_variant >= GRID_VARIANTS)
    return set_error(AFD_ERR_INVALID, "grid_variant must lie in -1..%d", GRID_VARIANTS - 1);
  if (o.offgrid_iters < 0 || o.offgrid_iters > 64)
    return set_error(AFD_ERR_INVALID, "offgrid_iters must lie in 0..64");
  if (o.offgrid_iters && o.renormalise)
    return set_error(AFD_ERR_INVALID, "offgrid_iters refines the plain objective: not with renormalise");
  return AFD_OK;
}

afd_status check_size(int N, int prec, bool allow_two_pass, bool allow_mixed) {
  if (allow_mixed && !is_pow2(N) && N >= (1 << MIN_LOGN)) {
    int radix[MIXED_MAX_PASSES];
    if (mixed_schedule(N, radix) < 2)
      return set_error(AFD_ERR_INVALID, "N = %d: must be a power of two or a product of powers of 2, 3, 5, 7, 11 and 13", N);
    if (mixed_smem_bytes(N, prec) > (size_t)MIXED_MAX_SMEM)
      return set_error(AFD_ERR_INVALID, "N = %d: largest mixed-radix size is %d for this precision", N,
                       (int)(MIXED_MAX_SMEM / (prec == AFD_FP32_GUARDED ? 16 : 32)));
    return AFD_OK;
  }
  if (!is_pow2(N) || N < (1 << MIN_LOGN))
    return set_error(AFD_ERR_INVALID,
                     allow_mixed ? "N = %d: must be >= 8 and a power of two or a product of powers of 2, 3, 5, 7, 11 and 13"
                                 : "N = %d: must be a power of two >= 8",
                     N);
  if (N > (1 << MAX_LOGN))
    return set_error(AFD_ERR_INVALID, "N = %d: largest supported power of two is %d", N, 1 << MAX_LOGN);
  if (!allow_two_pass && prec == AFD_FP32_GUARDED && N == (1 << TWO_PASS_LOGN))
    return set_error(AFD_ERR_INVALID, "N = %d in FP32 (the two-pass path) needs its own plan", N);
  return AFD_OK;
}

afd_status check_radii(const double* radii, int M) {
  if (!radii) return set_error(AFD_ERR_INVALID, "radii is NULL");
  if (M < 1 || M > 4096) return set_error(AFD_ERR_INVALID, "M = %d: must lie in 1..4096", M);
  for (int s = 0; s < M; ++s) {
    if (!(radii[s] >= 0.0 && radii[s] < 1.0))
      return set_error(AFD_ERR_INVALID, "radius %d = %g outside [0, 1)", s, radii[s]);
    if (s > 0 && !(radii[s] > radii[s - 1]))
      return set_error(AFD_ERR_INVALID, "radii must be strictly ascending (index %d)", s);
  }
  return AFD_OK;
}

afd_status resolve_opts(const afd_plan_opts* in, afd_plan_opts& o) {
  afd_plan_opts_default(&o);
  if (in) o = *in;
  return check_opts(o);
}

afd_status resolve_device(const afd_plan_opts& o, int& dev) {
  dev = o.device;
  if (dev < 0) CUDA_TRY(cudaGetDevice(&dev));
  int count = 0;
  CUDA_TRY(cudaGetDeviceCount(&count));
  if (dev >= count) return set_error(AFD_ERR_INVALID, "device %d not present (%d devices)", dev, count);
  return AFD_OK;
}

afd_status normalise_opts(const afd_plan_opts* in, afd_plan_opts& o, int& dev) {
  AFD_TRY(resolve_opts(in, o));
  return resolve_device(o, dev);
}

// ------------------------------------------------------------------ tables --

Tables::~Tables() {
  if (mem) cudaFree(mem);
  if (nu_mem) cudaFree(nu_mem);
}

afd_status Tables::build_nu(int nN_, const double* theta, const double* w, int L, const double* r, int M_) {
  AFD_TRY(build(L, r, M_, AFD_FP32_GUARDED));  // non-uniform plans: FP32 path, L <= 8192
  nu = true;
  nN = nN_;
  const double two_pi = 6.283185307179586476925286766559;
  // folds per radius: r^(P L) <= 2^-64
  std::vector<int> P(M);
  std::vector<float> rN32(M), wsq(M);
  int Pmax = 1;
  for (int s = 0; s < M; ++s) {
    const double rr = radii[s];
    int f = 1;
    if (rr > 0.0) f = (int)std::ceil(64.0 * std::log(2.0) / ((double)L * -std::log(rr)));
    f = std::max(f, 1);
    if (f > NU_MAX_FOLDS)
      return set_error(AFD_ERR_INVALID, "radius %g needs %d folds of %d angles (at most %d): use more angles", rr, f,
                       L, NU_MAX_FOLDS);
    P[s] = f;
    Pmax = std::max(Pmax, f);
    rN32[s] = (float)std::pow(rr, (double)L);
    wsq[s] = (float)((1.0 - rr) * (1.0 + rr));  // objective weight: (1 - r^2) |F|^2
  }
  nLc = Pmax * L;
  std::vector<double> z(2 * (size_t)nN), ww(nN);
  std::vector<unsigned long long> U(nN);
  for (int m = 0; m < nN; ++m) {
    z[2 * m] = std::cos(theta[m]);
    z[2 * m + 1] = std::sin(theta[m]);
    if (w) {
      ww[m] = w[m];
    } else {  // half the arc to each neighbour, cyclically
      const double nxt = m + 1 < nN ? theta[m + 1] : theta[0] + two_pi;
      const double prv = m > 0 ? theta[m - 1] : theta[nN - 1] - two_pi;
      ww[m] = (nxt - prv) / (2.0 * two_pi);
    }
    const double frac = theta[m] / two_pi;  // in [0, 1)
    U[m] = (unsigned long long)std::ldexp(frac, 64);
  }
  size_t off = 0;
  auto place = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
  const size_t o_z = place(16 * (size_t)nN), o_w = place(8 * (size_t)nN), o_U = place(8 * (size_t)nN),
               o_P = place(4 * (size_t)M), o_rN = place(4 * (size_t)M), o_wsq = place(4 * (size_t)M);
  CUDA_TRY(cudaMalloc(&nu_mem, off));
  bytes += off;
  char* b = static_cast<char*>(nu_mem);
  CUDA_TRY(cudaMemcpy(b + o_z, z.data(), 16 * (size_t)nN, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b + o_w, ww.data(), 8 * (size_t)nN, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b + o_U, U.data(), 8 * (size_t)nN, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b + o_P, P.data(), 4 * (size_t)M, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b + o_rN, rN32.data(), 4 * (size_t)M, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b + o_wsq, wsq.data(), 4 * (size_t)M, cudaMemcpyHostToDevice));
  dev.nN = nN;
  dev.nLc = nLc;
  dev.nz64 = reinterpret_cast<const double2*>(b + o_z);
  dev.nw64 = reinterpret_cast<const double*>(b + o_w);
  dev.nU = reinterpret_cast<const unsigned long long*>(b + o_U);
  dev.nP = reinterpret_cast<const int*>(b + o_P);
  dev.nrN32 = reinterpret_cast<const float*>(b + o_rN);
  dev.wsq32 = reinterpret_cast<const float*>(b + o_wsq);
  return AFD_OK;
}

// Shape of a plan's tables: the power-table split r^l = lo[l mod B] hi[l div B]
// (B = N / first radix), the stage-twiddle size of the power-of-two FFTs, and
// Shape of a plan's tables.  slog: log2 of the transforms the FFT stage
// twiddles serve (256-point sub-transforms on the two-pass path, the resident
// sub-transforms of a split size, else N); B: the split point of the radial
// powers r^l = lo[l mod B] hi[l div B]; tw32n: whether the FP32 twiddles w^k of
// all N points are needed (two-pass, split FP32 and mixed-radix transforms).
struct TableShape {
  int logN, B, H, tws, slog, ls;
  bool two_pass, mixed;
  int mix_npass;
  int mix_radix[MIXED_MAX_PASSES];
  TableShape(int N, int prec) {
    mixed = !is_pow2(N);
    logN = mixed ? -1 : ilog2(N);
    two_pass = !mixed && prec == AFD_FP32_GUARDED && logN == TWO_PASS_LOGN;
    ls = mixed || two_pass ? 0 : split_log(logN, prec);
    slog = two_pass ? 8 : logN - ls;
    mix_npass = mixed ? mixed_schedule(N, mix_radix) : 0;
    if (mixed) B = N / mix_radix[0];
    else B = two_pass ? 256 : FftSchedule::pow_b(slog);
    H = N / B;
    tws = mixed ? 1 : std::max(FftSchedule::tw_size(slog), 1);
  }
  bool tw32n() const { return two_pass || mixed || (ls > 0 && prec32); }
  bool prec32 = false;
};

size_t Tables::bytes_for(int N, int M, int prec) {
  TableShape sh(N, prec);
  sh.prec32 = prec == AFD_FP32_GUARDED;
  const int B = sh.B, H = sh.H;
  const size_t tws = (size_t)sh.tws;
  size_t off = 0;
  for (size_t b : {sizeof(double) * M, 16 * (size_t)N, 16 * tws, 8 * tws, 8 * tws, 8 * (size_t)M * B, 8 * (size_t)M * H,
                   4 * (size_t)M * B, 4 * (size_t)M * H, 4 * (size_t)M, 8 * (size_t)M, 8 * (size_t)M,
                   8 * (size_t)M, 4 * (size_t)M, 16 * (size_t)M * N, sh.tw32n() ? 8 * ((size_t)N + (sh.two_pass ? 4096 : 0)) : 0})
    off = align_up(off + b);
  return off;
}

afd_status Tables::build(int N_, const double* r, int M_, int prec_) {
    N = N_;
    M = M_;
    prec = prec_;
    radii.assign(r, r + M);
    TableShape sh(N, prec);
    sh.prec32 = prec == AFD_FP32_GUARDED;
    const int logN = sh.logN;
    const bool two_pass = sh.two_pass;
    // the two-pass path splits r^l at 256 and runs 256-point sub-transforms
    const int B = sh.B, H = sh.H;
    const int slog = sh.slog;  // log2 of the transforms the stage twiddles serve
    const int TWS = sh.mixed ? 0 : FftSchedule::tw_size(slog);
    std::vector<double> tw64(2 * (size_t)N), st64(2 * (size_t)std::max(TWS, 1)),
        rlo64((size_t)M * B), rhi64((size_t)M * H);
    std::vector<float> st32(2 * (size_t)std::max(TWS, 1)), rlo32((size_t)M * B), rhi32((size_t)M * H),
        wsq32(M);
    std::vector<double> w64(M), sq64(M), rho64(M);
    std::vector<float> rho32(M);
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < N; ++k) {
      // exact values at the quarter turns, libm elsewhere
      const double t = two_pi * (double)k / (double)N;
      double c = std::cos(t), sn = std::sin(t);
      if (4 * (long)k % N == 0) {
        const int q = (int)(4 * (long)k / N);
        c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
        sn = (q == 1) ? 1.0 : (q == 3 ? -1.0 : 0.0);
      }
      tw64[2 * k] = c;
      tw64[2 * k + 1] = sn;
    }
    // FFT stage twiddles of 2^slog-point transforms: pass p, input q, class k
    // -> exp(2 pi i q k / (ns R)) = w^(q k stride), w = exp(2 pi i / N)
    for (int p = 1; !sh.mixed && p < FftSchedule::npass(slog); ++p) {
      const int R = FftSchedule::radix(slog, p), NS = FftSchedule::ns(slog, p);
      const int off = FftSchedule::tw_off(slog, p), stride = N / (NS * R);
      for (int q = 1; q < R; ++q)
        for (int k = 0; k < NS; ++k) {
          const size_t e = (size_t)off + (size_t)(q - 1) * NS + k;
          const size_t src = (size_t)q * k * stride;
          st64[2 * e] = tw64[2 * src];
          st64[2 * e + 1] = tw64[2 * src + 1];
          st32[2 * e] = (float)tw64[2 * src];
          st32[2 * e + 1] = (float)tw64[2 * src + 1];
        }
    }
    for (int s = 0; s < M; ++s) {
      const double rr = radii[s];
      for (int q = 0; q < B; ++q) rlo64[(size_t)s * B + q] = std::pow(rr, (double)q);
      for (int h = 0; h < H; ++h) rhi64[(size_t)s * H + h] = std::pow(rr, (double)B * h);
      for (int q = 0; q < B; ++q) rlo32[(size_t)s * B + q] = (float)rlo64[(size_t)s * B + q];
      for (int h = 0; h < H; ++h) rhi32[(size_t)s * H + h] = (float)rhi64[(size_t)s * H + h];
      const double one_m_r2 = (1.0 - rr) * (1.0 + rr);
      const double one_m_rN = 1.0 - std::pow(rr, (double)N);
      sq64[s] = std::sqrt(one_m_r2);
      w64[s] = sq64[s] / one_m_rN;
      // 1 / ||e_a||_N^2 at a grid point: the aliased geometric series gives
      // ||e_a||_N^2 = (1 + r^N) / (1 - r^N)
      rho64[s] = one_m_rN / (2.0 - one_m_rN);
      rho32[s] = (float)rho64[s];
      wsq32[s] = (float)(one_m_r2 / (one_m_rN * one_m_rN));
    }
    // one allocation, 256-byte aligned sub-arrays (sizes as in Tables::bytes_for)
    size_t off = 0;
    auto place = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_r = place(sizeof(double) * M), o_tw64 = place(16 * (size_t)N),
                 o_st64 = place(8 * st64.size()), o_st32 = place(4 * st32.size()),
                 o_st32p = place(4 * st32.size()),
                 o_rlo64 = place(8 * rlo64.size()), o_rhi64 = place(8 * rhi64.size()),
                 o_rlo32 = place(4 * rlo32.size()), o_rhi32 = place(4 * rhi32.size()),
                 o_wsq = place(4 * (size_t)M), o_w64 = place(8 * (size_t)M), o_sq = place(8 * (size_t)M),
                 o_rho64 = place(8 * (size_t)M), o_rho32 = place(4 * (size_t)M), o_K = place(16 * (size_t)M * N),
                 o_tw32n = place(sh.tw32n() ? 8 * ((size_t)N + (sh.two_pass ? 4096 : 0)) : 0);
    CUDA_TRY(cudaMalloc(&mem, off));
    bytes = off;
    char* b = static_cast<char*>(mem);
    CUDA_TRY(cudaMemcpy(b + o_r, radii.data(), 8 * (size_t)M, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_tw64, tw64.data(), 16 * (size_t)N, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_st64, st64.data(), 8 * st64.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_st32, st32.data(), 4 * st32.size(), cudaMemcpyHostToDevice));
    {
      // entries 2j and 2j + 1 side by side per component (tw_size is even:
      // every pass after the first has an even ns)
      std::vector<float> st32p(st32.size(), 0.f);
      for (size_t j = 0; j + 1 < (size_t)TWS; j += 2) {
        st32p[2 * j] = st32[2 * j];
        st32p[2 * j + 1] = st32[2 * j + 2];
        st32p[2 * j + 2] = st32[2 * j + 1];
        st32p[2 * j + 3] = st32[2 * j + 3];
      }
      CUDA_TRY(cudaMemcpy(b + o_st32p, st32p.data(), 4 * st32p.size(), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(b + o_rlo64, rlo64.data(), 8 * rlo64.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_rhi64, rhi64.data(), 8 * rhi64.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_rlo32, rlo32.data(), 4 * rlo32.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_rhi32, rhi32.data(), 4 * rhi32.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_wsq, wsq32.data(), 4 * (size_t)M, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_w64, w64.data(), 8 * (size_t)M, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_sq, sq64.data(), 8 * (size_t)M, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_rho64, rho64.data(), 8 * (size_t)M, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b + o_rho32, rho32.data(), 4 * (size_t)M, cudaMemcpyHostToDevice));
    dev.N = N;
    dev.logN = logN;
    dev.ls = sh.ls;
    dev.M = M;
    dev.B = B;
    dev.radii = reinterpret_cast<const double*>(b + o_r);
    dev.tw64 = reinterpret_cast<const double2*>(b + o_tw64);
    dev.st64 = reinterpret_cast<const double2*>(b + o_st64);
    dev.st32 = reinterpret_cast<const float2*>(b + o_st32);
    dev.st32p = reinterpret_cast<const float4*>(b + o_st32p);
    dev.rlo64 = reinterpret_cast<const double*>(b + o_rlo64);
    dev.rhi64 = reinterpret_cast<const double*>(b + o_rhi64);
    dev.rlo32 = reinterpret_cast<const float*>(b + o_rlo32);
    dev.rhi32 = reinterpret_cast<const float*>(b + o_rhi32);
    dev.wsq32 = reinterpret_cast<const float*>(b + o_wsq);
    dev.w64 = reinterpret_cast<const double*>(b + o_w64);
    dev.sq64 = reinterpret_cast<const double*>(b + o_sq);
    dev.rho64 = reinterpret_cast<const double*>(b + o_rho64);
    dev.rho32 = reinterpret_cast<const float*>(b + o_rho32);
    dev.K64 = reinterpret_cast<const double2*>(b + o_K);
    dev.tw32n = nullptr;
    dev.inv_n = 1.0 / (double)N;
    dev.mix_npass = sh.mix_npass;
    for (int i = 0; i < MIXED_MAX_PASSES; ++i) dev.mix_radix[i] = i < sh.mix_npass ? sh.mix_radix[i] : 0;
    if (sh.tw32n()) {
      const size_t extra = two_pass ? 4096 : 0;  // exp(2 pi i m / 4096) = w^(16 m)
      std::vector<float> tw32n(2 * ((size_t)N + extra));
      for (size_t i = 0; i < 2 * (size_t)N; ++i) tw32n[i] = (float)tw64[i];
      for (size_t m = 0; m < extra; ++m) {
        tw32n[2 * (N + m)] = (float)tw64[2 * 16 * m];
        tw32n[2 * (N + m) + 1] = (float)tw64[2 * 16 * m + 1];
      }
      CUDA_TRY(cudaMemcpy(b + o_tw32n, tw32n.data(), 4 * tw32n.size(), cudaMemcpyHostToDevice));
      dev.tw32n = reinterpret_cast<const float2*>(b + o_tw32n);
    }
    CUDA_TRY(launch_kernel_table(dev.radii, M, N, reinterpret_cast<double2*>(b + o_K), nullptr));
    CUDA_TRY(cudaDeviceSynchronize());
    return AFD_OK;
}

}  // namespace afd

namespace {

// ------------------------------------------------------------- slot pools --

// Device buffers of n signals, pooled.  Signals are grouped by logN for
// launching; `ids_dev` holds, group after group, the slot indices.
struct SlotPool {
  int n = 0, K_max = 0, prec = 1, cap = 16;
  std::vector<SlotDev> host;        // descriptors (device pointers inside)
  std::vector<size_t> g_off;        // offset of signal i in the packed samples (doubles)
  size_t g_total = 0;               // packed sample count (doubles)
  void* mem = nullptr;
  SlotDev* slots_dev = nullptr;
  int* ids_dev = nullptr;
  StepRec* rec_dev = nullptr;       // n * K_max, signal-major
  SlotCtl* ctl_dev = nullptr;       // n
  size_t ctl_bytes = 0;             // control blocks and barrier counters
  double2* G_dev = nullptr;         // packed remainders
  StepRec* rec_host = nullptr;      // pinned mirrors
  bool rec_fresh = false;           // rec_host holds the last run's records
  std::vector<SlotDev> uploaded;    // the descriptors as last copied to slots_dev (empty: none)
  SlotCtl* ctl_host = nullptr;
  struct Group {
    int N, logN, first, count, Mmax;  // logN = -1: mixed-radix N
    bool nu;                          // non-uniform samples (single-signal plans)
    int nN, nLc;
    int variant = 0;                  // grid-kernel variant (autotuned for batches)
    float variant_us = 0.f;           // its measured time per launch (0: not tuned)
  };
  std::vector<Group> groups;
  std::vector<Fft2Maps> maps;       // TMA descriptors of two-pass slots (N = 65536)
  bool persistent = false;          // single FP32 slot: one persistent launch per decomposition
  int offgrid = 0;                  // off-grid refinement: Newton iterations per step (0: off)
  bool multi = false;               // batch: all signals in one multi-signal persistent launch
  unsigned* bar_dev = nullptr;      // grid-barrier counter and error word (BAR_BYTES, in the ctl area)
  MultiArgs margs{};                // the multi-signal launch's arguments

  ~SlotPool() { release(); }
  void release() {
    if (mem) cudaFree(mem);
    if (rec_host) cudaFreeHost(rec_host);
    if (ctl_host) cudaFreeHost(ctl_host);
    mem = nullptr;
    rec_host = nullptr;
    ctl_host = nullptr;
    rec_fresh = false;
    uploaded.clear();
  }

  // tables[i] is the plan of signal i.
  // allow_multi: a batch that may run as one multi-signal persistent launch.
  afd_status build(const std::vector<const Tables*>& tables, int K, const afd_plan_opts& o, bool allow_multi = false) {
    release();
    n = (int)tables.size();
    K_max = K;
    prec = o.precision;
    offgrid = o.offgrid_iters;
    persistent = o.persistent != 0 && offgrid == 0;
    cap = prec == AFD_FP32_GUARDED ? o.guard_cap : 1;
    // group by N (stable: signal order within a group)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return tables[a]->N < tables[b]->N; });
    groups.clear();
    for (int idx = 0; idx < n; ++idx) {
      const int i = order[idx];
      const Tables& T = *tables[i];
      const int Ni = T.N;
      if (groups.empty() || groups.back().N != Ni || groups.back().nu != T.nu)
        groups.push_back({Ni, is_pow2(Ni) ? ilog2(Ni) : -1, idx, 0, 0, T.nu, T.nN, T.nLc, 0, 0.f});
      groups.back().count++;
      groups.back().Mmax = std::max(groups.back().Mmax, tables[i]->M);
    }
    for (auto& g : groups)
      if (o.grid_variant >= 0 && grid_variant_ok(g.logN, prec, o.grid_variant)) g.variant = o.grid_variant;
    // sizes
    g_off.assign(n, 0);
    g_total = 0;
    for (int i = 0; i < n; ++i) {
      g_off[i] = g_total;
      g_total += 2 * (size_t)tables[i]->samples();
    }
    size_t off = 0;
    auto place = [&](size_t bytes) { size_t o2 = off; off = align_up(off + bytes); return o2; };
    const size_t o_G = place(8 * g_total);
    std::vector<size_t> o_c(n), o_g32(n), o_top(n), o_cand(n), o_gp(n), o_ep(n), o_X(n), o_G2(n), o_g32b(n),
        o_rf(n);
    for (int i = 0; i < n; ++i) {
      const int N = tables[i]->samples(), M = tables[i]->M;
      const bool two_pass = !tables[i]->nu && prec && N == (1 << TWO_PASS_LOGN);
      // best pairs per radius: one per pass-2 row block (two-pass), one per
      // sub-transform (split sizes), else one
      const size_t per_radius = two_pass ? 16 : (size_t)1 << tables[i]->dev.ls;
      o_c[i] = place((prec ? 8 : 16) * (size_t)tables[i]->spectrum());
      o_g32[i] = place(prec ? 8 * (size_t)N : 0);
      // the persistent kernel alternates two remainder buffers and two FP32 copies
      o_G2[i] = place(persistent ? 16 * (size_t)N : 0);
      o_g32b[i] = place(persistent && prec ? 8 * (size_t)N : 0);
      o_X[i] = place(two_pass ? 8 * (size_t)M * N : 0);
      // two-pass: one best pair per (radius, 16-row block of pass 2)
      o_top[i] = place((prec ? sizeof(Top2F) : sizeof(Top2D)) * (size_t)M * per_radius);
      o_cand[i] = place(sizeof(int2) * cap);
      // the persistent kernel keeps one partial per 32-sample warp item, and
      // its energy partials for every step
      const size_t parts = (size_t)chunks_of(N) * (persistent ? FP64_CHUNK / 32 : 1);
      o_gp[i] = place(sizeof(double2) * cap * parts);
      o_ep[i] = place(sizeof(double) * parts * (persistent ? (size_t)K_max : 1));
      o_rf[i] = place(offgrid ? sizeof(double) * 2 * RF_MAX_CTAS * 6 : 0);
    }
    const size_t o_rec = place(sizeof(StepRec) * (size_t)n * K_max);
    // control blocks, then the grid-barrier counter and error word of the
    // persistent kernels; one memset per run clears both
    ctl_bytes = align_up(sizeof(SlotCtl) * (size_t)n) + BAR_BYTES;
    const size_t o_ctl = place(ctl_bytes);
    const size_t o_slots = place(sizeof(SlotDev) * (size_t)n);
    const size_t o_ids = place(sizeof(int) * (size_t)n);
    CUDA_TRY(cudaMalloc(&mem, off));
    CUDA_TRY(cudaMemset(mem, 0, off));
    CUDA_TRY(cudaMallocHost((void**)&rec_host, sizeof(StepRec) * (size_t)n * K_max));
    CUDA_TRY(cudaMallocHost((void**)&ctl_host, sizeof(SlotCtl) * (size_t)n));
    char* b = static_cast<char*>(mem);
    G_dev = reinterpret_cast<double2*>(b + o_G);
    rec_dev = reinterpret_cast<StepRec*>(b + o_rec);
    ctl_dev = reinterpret_cast<SlotCtl*>(b + o_ctl);
    slots_dev = reinterpret_cast<SlotDev*>(b + o_slots);
    ids_dev = reinterpret_cast<int*>(b + o_ids);
    host.assign(n, SlotDev{});
    for (int i = 0; i < n; ++i) {
      SlotDev& d = host[i];
      d.p = tables[i]->dev;
      d.K_max = K_max;
      d.prec = prec;
      d.cap = cap;
      d.force_a1_zero = o.force_a1_zero;
      d.renorm = o.renormalise != 0;
      d.tol = 0.0;
      d.tau = o.guard_tau;
      d.G = reinterpret_cast<double2*>(b + o_G) + g_off[i] / 2;
      d.c32 = prec ? reinterpret_cast<float2*>(b + o_c[i]) : nullptr;
      d.g32 = prec ? reinterpret_cast<float2*>(b + o_g32[i]) : nullptr;
      d.G2 = persistent ? reinterpret_cast<double2*>(b + o_G2[i]) : nullptr;
      d.g32b = persistent && prec ? reinterpret_cast<float2*>(b + o_g32b[i]) : nullptr;
      d.X = !tables[i]->nu && prec && tables[i]->N == (1 << TWO_PASS_LOGN) ? reinterpret_cast<float2*>(b + o_X[i])
                                                                            : nullptr;
      d.c64 = prec ? nullptr : reinterpret_cast<double2*>(b + o_c[i]);
      d.top2 = b + o_top[i];
      d.cand = reinterpret_cast<int2*>(b + o_cand[i]);
      d.gpart = reinterpret_cast<double2*>(b + o_gp[i]);
      d.rfpart = offgrid ? reinterpret_cast<double*>(b + o_rf[i]) : nullptr;
      d.epart = reinterpret_cast<double*>(b + o_ep[i]);
      d.rec = rec_dev + (size_t)i * K_max;
      d.ctl = ctl_dev + i;
      d.bar = reinterpret_cast<unsigned*>(b + o_ctl + align_up(sizeof(SlotCtl) * (size_t)n));
    }
    CUDA_TRY(cudaMemcpy(ids_dev, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    bar_dev = reinterpret_cast<unsigned*>(b + o_ctl + align_up(sizeof(SlotCtl) * (size_t)n));
    // The multi-signal persistent kernel takes a batch when every signal is an
    // FP32-path power of two it holds on chip or of a mixed-radix size (not
    // beside N = 16384).  Not a single signal of a mixed-radix size: there the
    // per-step kernels measured faster (0.70 ms against 0.93-1.31 ms at
    // N = 3000; the kernel's FP64 items are made for many signals).
    multi = allow_multi && n > 1 && prec == AFD_FP32_GUARDED && (int)groups.size() <= MULTI_MAX_CLASSES;
    bool any_mixed = false, any_big = false;
    for (const auto& g : groups) {
      multi = multi && !g.nu && (g.logN > 0 ? multi_size_ok(g.logN) : g.logN < 0);
      any_mixed = any_mixed || g.logN < 0;
      any_big = any_big || g.logN > 13;
    }
    // mixed-radix items run in the 256-thread build, which N = 16384 leaves
    if (any_mixed && any_big) multi = false;
    margs = MultiArgs{};
    if (multi) {
      margs.slots = slots_dev;
      margs.ids = ids_dev;
      margs.fresh_ids = ids_dev;
      margs.bar = bar_dev;
      margs.K = K;
      margs.final_forward = 0;
      margs.n_cls = margs.n_fresh = (int)groups.size();
      for (size_t gi = 0; gi < groups.size(); ++gi) {
        MultiClass& c = margs.cls[gi];
        if (groups[gi].logN < 0) multi_class_shape_mixed(groups[gi].N, groups[gi].Mmax, groups[gi].count, cap, &c);
        else multi_class_shape(groups[gi].logN, groups[gi].Mmax, groups[gi].count, cap, &c);
        c.first = groups[gi].first;
        margs.fresh[gi] = c;
      }
    }
    maps.assign(n, Fft2Maps{});
    for (int i = 0; i < n; ++i) {
      if (!host[i].X) continue;
      const int r = fft2_make_maps(&maps[i], host[i].c32, host[i].g32, host[i].X, tables[i]->M);
      if (r) return set_error(AFD_ERR_CUDA, "tensor map encoding failed (driver status %d)", r);
    }
    return upload(0.0, nullptr);
  }

  // Copies the descriptors to the device unless they equal what is there:
  // only build() and this function write slots_dev.
  afd_status upload(double tol, cudaStream_t st) {
    for (auto& d : host) d.tol = tol;
    if (uploaded.size() == host.size() && std::memcmp(uploaded.data(), host.data(), sizeof(SlotDev) * n) == 0)
      return AFD_OK;
    uploaded.clear();
    if (st) {
      CUDA_TRY(cudaMemcpyAsync(slots_dev, host.data(), sizeof(SlotDev) * n, cudaMemcpyHostToDevice, st));
    } else {
      CUDA_TRY(cudaMemcpy(slots_dev, host.data(), sizeof(SlotDev) * n, cudaMemcpyHostToDevice));
    }
    uploaded = host;
    return AFD_OK;
  }
};

// Kernel launch bookkeeping.  Kernel kinds: 0 grid, 1 guard, 2 update,
// 3 forward, 4 persistent (initialisation is not timed).
constexpr int KINDS = 5;  // + 4: the persistent whole-decomposition kernel
struct Counters {
  long long launches = 0;
  long long n[KINDS] = {};
  double ms[KINDS] = {};
};

// Optional CUDA-event timing of every kernel of the step sequence.  Events are
// recorded between consecutive kernels on their stream; under stream capture
// they become event-record nodes of the graph, so a replayed graph is timed
// as it runs.
struct StepTimer {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;  // kind of the kernel that ends at event i; -1 opens a sequence
  size_t used = 0;
  ~StepTimer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  afd_status mark(cudaStream_t st, int k) {
    if (!on) return AFD_OK;
    if (ev.size() <= used) {
      cudaEvent_t e;
      CUDA_TRY(cudaEventCreate(&e));
      ev.push_back(e);
      kind.push_back(k);
    }
    kind[used] = k;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusActive) {
      CUDA_TRY(cudaEventRecordWithFlags(ev[used], st, cudaEventRecordExternal));
    } else {
      CUDA_TRY(cudaEventRecord(ev[used], st));
    }
    ++used;
    return AFD_OK;
  }
  // Events of the last run (or of the captured graph) after the stream has
  // been synchronised.
  afd_status collect(Counters& c, size_t count) {
    for (size_t i = 1; i < count; ++i) {
      if (kind[i] < 0 || kind[i] >= KINDS) continue;
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, ev[i - 1], ev[i]));
      c.ms[kind[i]] += ms;
    }
    return AFD_OK;
  }
};

// Enqueue the initialisation and K greedy steps of one group on stream st.
afd_status enqueue_group(const SlotPool& pool, const SlotPool::Group& g, int K, cudaStream_t st,
                         Counters& cnt, StepTimer* timer) {
  const SlotDev* slots = pool.slots_dev;
  const int* ids = pool.ids_dev + g.first;
  const int prec = pool.prec;
  const bool t = timer && timer->on;
  // the two-pass path (N = 65536) serves single-signal plans: slot 0
  if (g.nu) {
    // non-uniform samples: init, non-uniform DFT, then per step grid, guard,
    // update and the next non-uniform DFT
    CUDA_TRY(launch_update_nu(slots, ids, g.nN, true, st));
    CUDA_TRY(launch_nudft(slots, ids, g.nLc, st));
    cnt.launches += 2;
    if (t) AFD_TRY(timer->mark(st, -1));
    for (int k = 0; k < K; ++k) {
      CUDA_TRY(launch_grid_nu(slots, ids, g.logN, g.Mmax, st));
      if (t) AFD_TRY(timer->mark(st, 0));
      CUDA_TRY(launch_guard_nu(slots, ids, g.nN, pool.cap, st));
      if (t) AFD_TRY(timer->mark(st, 1));
      CUDA_TRY(launch_update_nu(slots, ids, g.nN, false, st));
      if (t) AFD_TRY(timer->mark(st, 2));
      cnt.n[0] += 1;
      cnt.n[1] += 1;
      cnt.n[2] += 1;
      cnt.launches += 3;
      if (k + 1 < K) {
        CUDA_TRY(launch_nudft(slots, ids, g.nLc, st));
        if (t) AFD_TRY(timer->mark(st, 3));
        cnt.n[3] += 1;
        cnt.launches += 1;
      }
    }
    return AFD_OK;
  }
  const bool two_pass = prec == AFD_FP32_GUARDED && g.logN == TWO_PASS_LOGN;
  const bool mixed = g.logN < 0;
  if (two_pass && (g.count != 1 || pool.n != 1)) return set_error(AFD_ERR_INVALID, "N = 65536 needs its own plan");
  const int per = two_pass ? 2 : 1;  // launches per transform stage
  if (pool.persistent && pool.n == 1 && prec == AFD_FP32_GUARDED && !mixed && g.logN <= PERSISTENT_MAX_LOGN) {
    CUDA_TRY(launch_init(slots, ids, g.count, g.N, st));
    if (t) AFD_TRY(timer->mark(st, -1));
    CUDA_TRY(launch_persistent(slots, g.logN, g.Mmax, st));
    if (t) AFD_TRY(timer->mark(st, 4));
    cnt.n[4] += 1;
    cnt.launches += 2;
    return AFD_OK;
  }
  auto forward = [&]() -> cudaError_t {
    if (two_pass) return launch_forward2(slots, pool.maps[0], st);
    if (mixed) return launch_forward_mixed(slots, ids, g.count, g.N, prec, st);
    return launch_forward(slots, ids, g.count, g.logN, prec, st);
  };
  CUDA_TRY(launch_init(slots, ids, g.count, g.N, st));
  CUDA_TRY(forward());
  cnt.launches += 1 + per;
  if (t) AFD_TRY(timer->mark(st, -1));
  for (int k = 0; k < K; ++k) {
    if (two_pass) CUDA_TRY(launch_grid2(slots, pool.maps[0], g.Mmax, st));
    else if (mixed) CUDA_TRY(launch_grid_mixed(slots, ids, g.count, g.N, prec, g.Mmax, st));
    else CUDA_TRY(launch_grid(slots, ids, g.count, g.logN, prec, g.Mmax, st, g.variant));
    if (t) AFD_TRY(timer->mark(st, 0));
    cnt.n[0] += per;
    cnt.launches += per;
    if (prec == AFD_FP32_GUARDED) {
      CUDA_TRY(launch_guard(slots, ids, g.count, g.N, pool.cap, st));
      if (t) AFD_TRY(timer->mark(st, 1));
      cnt.n[1] += 1;
      cnt.launches += 1;
    }
    if (pool.offgrid > 0) {
      // the winner refined off the grid, then the general update
      CUDA_TRY(launch_refine(slots, ids, g.count, g.N, pool.offgrid, st));
      CUDA_TRY(launch_update_offgrid(slots, ids, g.count, g.N, st));
      cnt.launches += 2;
    } else {
      CUDA_TRY(launch_update(slots, ids, g.count, g.N, st));
      cnt.launches += 1;
    }
    if (t) AFD_TRY(timer->mark(st, 2));
    cnt.n[2] += 1;
    if (k + 1 < K) {
      CUDA_TRY(forward());
      if (t) AFD_TRY(timer->mark(st, 3));
      cnt.n[3] += per;
      cnt.launches += per;
    }
  }
  return AFD_OK;
}

// --------------------------------------------------------------- autotuner --
//
// A batch chooses, per N-class, among the bitwise-equivalent grid-kernel
// variants (points per thread, CTA width) by timing each on the batch's own
// first step: the group's slots are initialised and transformed, then in
// each of kTuneRounds rounds every variant runs one warm-up and kTuneReps
// timed launches (CUDA events on the batch's stream); the variant with the
// fastest round is kept.  Choices are cached per process by
// (device, N, radii count, signal count), so later batches of the same shape
// skip the measurement.
constexpr int kTuneReps = 3;
constexpr int kTuneRounds = 3;  // interleaved rounds over the variants
std::mutex g_tune_mu;
std::map<std::array<int, 4>, std::pair<int, float>> g_tune_cache;

afd_status autotune(SlotPool& pool, int device, cudaStream_t st) {
  if (pool.multi) return AFD_OK;  // the multi-signal kernel has one grid variant per size
  for (auto& g : pool.groups) {
    if (g.nu || g.logN < 0 || g.logN > MAX_LOGN_RESIDENT || pool.prec != AFD_FP32_GUARDED) continue;
    int n_ok = 0;
    for (int v = 0; v < GRID_VARIANTS; ++v) n_ok += grid_variant_ok(g.logN, pool.prec, v) ? 1 : 0;
    if (n_ok < 2) continue;
    const std::array<int, 4> key{device, g.N, g.Mmax, g.count};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        g.variant = it->second.first;
        g.variant_us = it->second.second;
        continue;
      }
    }
    const int* ids = pool.ids_dev + g.first;
    CUDA_TRY(cudaMemsetAsync(pool.ctl_dev, 0, sizeof(SlotCtl) * pool.n, st));
    CUDA_TRY(launch_init(pool.slots_dev, ids, g.count, g.N, st));
    CUDA_TRY(launch_forward(pool.slots_dev, ids, g.count, g.logN, pool.prec, st));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // Rounds over all variants, each variant's best round counts: a
    // variant timed while the clocks ramp up or another process runs is not
    // chosen or dropped for that alone.
    float var_us[GRID_VARIANTS];
    for (int v = 0; v < GRID_VARIANTS; ++v) var_us[v] = 3.0e38f;
    cudaError_t err = cudaSuccess;
    for (int round = 0; round < kTuneRounds && err == cudaSuccess; ++round) {
      for (int v = 0; v < GRID_VARIANTS && err == cudaSuccess; ++v) {
        if (!grid_variant_ok(g.logN, pool.prec, v)) continue;
        err = launch_grid(pool.slots_dev, ids, g.count, g.logN, pool.prec, g.Mmax, st, v);
        if (err == cudaSuccess) err = cudaEventRecord(e0, st);
        for (int r = 0; r < kTuneReps && err == cudaSuccess; ++r)
          err = launch_grid(pool.slots_dev, ids, g.count, g.logN, pool.prec, g.Mmax, st, v);
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess) var_us[v] = std::min(var_us[v], 1e3f * ms / kTuneReps);
      }
    }
    int best = 0;
    float best_us = var_us[0];
    for (int v = 1; v < GRID_VARIANTS; ++v)
      if (grid_variant_ok(g.logN, pool.prec, v) && var_us[v] < best_us) {
        best = v;
        best_us = var_us[v];
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "autotune", __LINE__);
    g.variant = best;
    g.variant_us = best_us;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {best, best_us};
  }
  return AFD_OK;
}

// Runs the whole K-step sequence for every group of the pool: groups on
// their own streams (forked from and joined back to `main`).
struct Runner {
  cudaStream_t main = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaEvent_t order = nullptr;  // orders a plan-owned stream after the legacy default stream
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_K = -1;
  bool graph_timed = false;
  size_t graph_events = 0;
  Counters graph_cnt;  // launches of one replay

  ~Runner() { destroy(); }
  // Drops the captured graph (the launch sequence changed).
  void destroy_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    graph_K = -1;
  }
  void destroy() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    graph_K = -1;
    for (auto s : side) cudaStreamDestroy(s);
    for (auto e : join) cudaEventDestroy(e);
    side.clear();
    join.clear();
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
    if (order) cudaEventDestroy(order);
    order = nullptr;
  }

  // A plan-owned stream does not synchronise with the legacy default stream,
  // so work the caller queued there (e.g. a copy producing G) is waited for.
  afd_status order_after_default() {
    if (!order) CUDA_TRY(cudaEventCreateWithFlags(&order, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(order, cudaStreamLegacy));
    CUDA_TRY(cudaStreamWaitEvent(main, order, 0));
    return AFD_OK;
  }

  afd_status prepare(size_t ngroups) {
    if (!fork) CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    while (side.size() + 1 < ngroups) {
      cudaStream_t s;
      cudaEvent_t e;
      CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      side.push_back(s);
      join.push_back(e);
    }
    return AFD_OK;
  }

  afd_status enqueue(const SlotPool& pool, int K, Counters& cnt, StepTimer* timer) {
    AFD_TRY(prepare(pool.groups.size()));
    if (timer) timer->used = 0;
    CUDA_TRY(cudaMemsetAsync(pool.ctl_dev, 0, pool.ctl_bytes, main));
    if (pool.multi) {
      // every signal of the batch, all K steps: one cooperative launch
      MultiArgs a = pool.margs;
      a.K = K;
      if (timer && timer->on) AFD_TRY(timer->mark(main, -1));
      CUDA_TRY(launch_multi(a, main));
      if (timer && timer->on) AFD_TRY(timer->mark(main, 4));
      cnt.n[4] += 1;
      cnt.launches += 1;
      return AFD_OK;
    }
    if (pool.groups.size() > 1) CUDA_TRY(cudaEventRecord(fork, main));
    for (size_t gi = 0; gi < pool.groups.size(); ++gi) {
      cudaStream_t st = gi == 0 ? main : side[gi - 1];
      if (gi > 0) CUDA_TRY(cudaStreamWaitEvent(st, fork, 0));
      AFD_TRY(enqueue_group(pool, pool.groups[gi], K, st, cnt, timer));
      if (gi > 0) {
        CUDA_TRY(cudaEventRecord(join[gi - 1], st));
        CUDA_TRY(cudaStreamWaitEvent(main, join[gi - 1], 0));
      }
    }
    return AFD_OK;
  }

  // Either replays a cached graph of the K-step sequence or launches directly;
  // with the timer on, per-kernel device times of this run are added to cnt.
  afd_status run(const SlotPool& pool, int K, bool use_graph, Counters& cnt, StepTimer* timer) {
    const bool timed = timer && timer->on;
    if (!use_graph) {
      AFD_TRY(enqueue(pool, K, cnt, timer));
      if (timed) {
        CUDA_TRY(cudaStreamSynchronize(main));
        AFD_TRY(timer->collect(cnt, timer->used));
      }
      return AFD_OK;
    }
    if (graph_K != K || graph_timed != timed) {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      exec = nullptr;
      graph = nullptr;
      graph_K = -1;
      Counters c2;
      CUDA_TRY(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
      afd_status st = enqueue(pool, K, c2, timer);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(main, &g);
      if (st != AFD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      CUDA_TRY(e);
      graph = g;
      CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
      graph_K = K;
      graph_timed = timed;
      graph_events = timed ? timer->used : 0;
      graph_cnt = c2;
    }
    CUDA_TRY(cudaGraphLaunch(exec, main));
    cnt.launches += graph_cnt.launches;
    for (int i = 0; i < KINDS; ++i) cnt.n[i] += graph_cnt.n[i];
    if (timed) {
      CUDA_TRY(cudaStreamSynchronize(main));
      AFD_TRY(timer->collect(cnt, graph_events));
    }
    return AFD_OK;
  }
};

}  // namespace

// ------------------------------------------------------------------- plans --

struct afd_plan {
  int device = 0;
  afd_plan_opts opts{};
  bool own_stream = false;
  Tables tables;
  SlotPool pool;
  Runner runner;
  Counters cnt;
  StepTimer timer;
  int last_steps = 0;
  long long* phase_dev = nullptr;  // persistent kernel phase stamps while profiling
  int phase_cap = 0;
  double phase_sum[7] = {};
  long long phase_steps = 0;
  ~afd_plan() {
    runner.destroy();
    if (own_stream && runner.main) cudaStreamDestroy(runner.main);
    if (phase_dev) cudaFree(phase_dev);
  }
};

struct afd_batch {
  int device = 0;
  afd_plan_opts opts{};
  bool own_stream = false;
  bool tuned = false;
  std::vector<std::unique_ptr<Tables>> tables;
  SlotPool pool;
  Runner runner;
  Counters cnt;
  std::vector<int> N;
  ~afd_batch() {
    runner.destroy();
    if (own_stream && runner.main) cudaStreamDestroy(runner.main);
  }
};

namespace {

// Whether the current device can write p directly (device or managed memory).
bool device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
template <typename T> T* dev_or_null(T* p) { return device_ptr(p) ? p : nullptr; }
template <typename T> T* host_or_null(T* p) { return device_ptr(p) ? nullptr : p; }

// Device-resident outputs are written by a gather kernel on the call's
// stream, straight from the step records (no host round trip); host ones are
// filled from the fetched records afterwards.  Returns whether any was on the
// device.
afd_status gather_device_outputs(const SlotPool& pool, int K_stride, double* a_out, double* coeff_out,
                                 double* delta_out, int* idx_out, int* steps_out, double* E1_out, cudaStream_t st) {
  double *a = dev_or_null(a_out), *c = dev_or_null(coeff_out), *d = dev_or_null(delta_out),
         *e = dev_or_null(E1_out);
  int *ix = dev_or_null(idx_out), *so = dev_or_null(steps_out);
  if (a || c || d || e || ix || so)
    CUDA_TRY(launch_gather(pool.rec_dev, pool.ctl_dev, pool.n, pool.K_max, K_stride, a, c, d, ix, so, e, st));
  return AFD_OK;
}

// Gather the records of signal i (steps = its step count) into caller host
// arrays (device ones are written by gather_device_outputs).
afd_status write_outputs(const SlotPool& pool, int i, int K_stride, int steps, double* a_out,
                         double* coeff_out, double* delta_out, int* idx_out) {
  const StepRec* r = pool.rec_host + (size_t)i * pool.K_max;
  std::vector<double> a(2 * (size_t)steps), c(2 * (size_t)steps), d((size_t)steps + 1);
  std::vector<int> ix(2 * (size_t)steps);
  const SlotCtl& ctl = pool.ctl_host[i];
  // delta_0: 1 for a fresh start, E(start) / E_1 for a resumed one
  d[0] = (ctl.E1 > 0.0 && ctl.Estart != ctl.E1) ? ctl.Estart / ctl.E1 : 1.0;
  for (int k = 0; k < steps; ++k) {
    a[2 * k] = r[k].a_re;
    a[2 * k + 1] = r[k].a_im;
    c[2 * k] = r[k].c_re;
    c[2 * k + 1] = r[k].c_im;
    d[k + 1] = r[k].delta;
    ix[2 * k] = r[k].s;
    ix[2 * k + 1] = r[k].j;
  }
  const size_t base2 = 2 * (size_t)i * K_stride, based = (size_t)i * (K_stride + 1);
  if (a_out) std::memcpy(a_out + base2, a.data(), 8 * a.size());
  if (coeff_out) std::memcpy(coeff_out + base2, c.data(), 8 * c.size());
  if (delta_out) std::memcpy(delta_out + based, d.data(), 8 * d.size());
  if (idx_out) std::memcpy(idx_out + base2, ix.data(), 4 * ix.size());
  return AFD_OK;
}

// The control blocks and, with_rec, the step records into the pinned mirrors
// (callers whose outputs are all on the device need only the control blocks;
// the records follow on demand, fetch_records).
afd_status fetch_results(SlotPool& pool, cudaStream_t st, bool with_rec) {
  pool.rec_fresh = false;
  if (with_rec)
    CUDA_TRY(cudaMemcpyAsync(pool.rec_host, pool.rec_dev, sizeof(StepRec) * (size_t)pool.n * pool.K_max,
                             cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(pool.ctl_host, pool.ctl_dev, sizeof(SlotCtl) * (size_t)pool.n,
                           cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  pool.rec_fresh = with_rec;
  return AFD_OK;
}
afd_status fetch_records(SlotPool& pool) {
  if (pool.rec_fresh || !pool.rec_host) return AFD_OK;
  CUDA_TRY(cudaMemcpy(pool.rec_host, pool.rec_dev, sizeof(StepRec) * (size_t)pool.n * pool.K_max,
                      cudaMemcpyDeviceToHost));
  pool.rec_fresh = true;
  return AFD_OK;
}

}  // namespace

extern "C" {

void afd_plan_opts_default(afd_plan_opts* o) {
  if (!o) return;
  o->precision = AFD_FP32_GUARDED;
  o->guard_tau = 1e-4;
  o->renormalise = 0;
  o->autotune = 1;
  o->grid_variant = -1;
  o->offgrid_iters = 0;
  o->guard_cap = 16;
  o->force_a1_zero = 0;
  o->device = -1;
  o->stream = nullptr;
  o->use_graph = 1;
  o->persistent = 1;
}

const char* afd_status_str(afd_status s) {
  switch (s) {
    case AFD_OK: return "AFD_OK";
    case AFD_PENDING: return "AFD_PENDING";
    case AFD_ERR_INVALID: return "AFD_ERR_INVALID";
    case AFD_ERR_NOMEM: return "AFD_ERR_NOMEM";
    case AFD_ERR_CUDA: return "AFD_ERR_CUDA";
    case AFD_ERR_TIMEOUT: return "AFD_ERR_TIMEOUT";
    case AFD_ERR_BUDGET: return "AFD_ERR_BUDGET";
    case AFD_ERR_NOT_FOUND: return "AFD_ERR_NOT_FOUND";
    case AFD_ERR_NUMERIC: return "AFD_ERR_NUMERIC";
  }
  return "AFD_UNKNOWN_STATUS";
}

const char* afd_last_error(void) { return last_error_text(); }

const char* afd_version(void) { return "0.1.0"; }

afd_status afd_selftest_wait_timeout(int device, int kind, afd_status* status, double* seconds) {
  clear_last_error();
  if (!status || !seconds) return set_error(AFD_ERR_INVALID, "status and seconds must not be NULL");
  if (kind != 0 && kind != 1) return set_error(AFD_ERR_INVALID, "kind %d: 0 (grid barrier) or 1 (mbarrier)", kind);
  int dev = device;
  if (dev < 0) CUDA_TRY(cudaGetDevice(&dev));
  DeviceScope scope(dev);
  if (!scope.ok) return set_error(AFD_ERR_INVALID, "cannot select device %d", dev);
  // one allocation: SlotCtl, the barrier counter and the timer (a 128-byte
  // line each), then the SlotDev that points at the first two
  constexpr size_t kBar = 128, kNs = 256, kSlot = 384;
  unsigned char* mem = nullptr;
  CUDA_TRY(cudaMalloc(&mem, kSlot + sizeof(SlotDev)));
  cudaStream_t st = nullptr;
  SlotDev h{};
  h.ctl = reinterpret_cast<SlotCtl*>(mem);
  h.bar = reinterpret_cast<unsigned*>(mem + kBar);
  SlotCtl ctl{};
  unsigned long long ns = 0;
  auto* d_ns = reinterpret_cast<unsigned long long*>(mem + kNs);
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(mem, 0, kSlot, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mem + kSlot, &h, sizeof(h), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = kind == 0 ? launch_selftest_barrier(reinterpret_cast<const SlotDev*>(mem + kSlot), d_ns, st)
                  : launch_selftest_mbarrier(h.ctl, d_ns, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, mem, sizeof(ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  afd_status rc = e == cudaSuccess ? AFD_OK : cuda_fail(e, "wait self-test", __LINE__);
  if (st) cudaStreamDestroy(st);
  cudaFree(mem);
  if (rc != AFD_OK) return rc;
  *status = (ctl.err & 4) ? AFD_ERR_TIMEOUT : AFD_OK;
  *seconds = 1e-9 * (double)ns;
  return AFD_OK;
}

afd_status afd_plan_create(afd_plan** out, int N, const double* radii, int M, const afd_plan_opts* opts) {
  clear_last_error();
  if (!out) return set_error(AFD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  afd_plan_opts o;
  int dev = 0;
  // every argument is checked before the first CUDA call
  AFD_TRY(resolve_opts(opts, o));
  AFD_TRY(check_size(N, o.precision, true, true));
  AFD_TRY(check_radii(radii, M));
  if (o.force_a1_zero && radii[0] != 0.0)
    return set_error(AFD_ERR_INVALID, "force_a1_zero needs radii[0] == 0");
  AFD_TRY(resolve_device(o, dev));
  DeviceScope scope(dev);
  if (!scope.ok) return set_error(AFD_ERR_CUDA, "cannot make device %d current", dev);
  AFD_TRY(ensure_configured(dev));
  std::unique_ptr<afd_plan> p(new (std::nothrow) afd_plan());
  if (!p) return set_error(AFD_ERR_NOMEM, "host allocation failed");
  p->device = dev;
  p->opts = o;
  if (o.stream) {
    p->runner.main = static_cast<cudaStream_t>(o.stream);
  } else {
    CUDA_TRY(cudaStreamCreateWithFlags(&p->runner.main, cudaStreamNonBlocking));
    p->own_stream = true;
  }
  AFD_TRY(p->tables.build(N, radii, M, o.precision));
  *out = p.release();
  return AFD_OK;
}

afd_status afd_plan_create_nonuniform(afd_plan** out, int N, const double* theta, const double* weights, int L,
                                      const double* radii, int M, const afd_plan_opts* opts) {
  clear_last_error();
  if (!out) return set_error(AFD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  afd_plan_opts o;
  int dev = 0;
  // every argument is checked before the first CUDA call
  AFD_TRY(resolve_opts(opts, o));
  if (o.precision != AFD_FP32_GUARDED)
    return set_error(AFD_ERR_INVALID, "non-uniform samples: the FP32-guarded path only");
  if (o.force_a1_zero || o.renormalise || o.offgrid_iters)
    return set_error(AFD_ERR_INVALID,
                     "non-uniform samples: force_a1_zero, renormalise and offgrid_iters are not supported");
  if (N < 1 || N > (1 << 20) || !theta) return set_error(AFD_ERR_INVALID, "need 1 <= N <= 2^20 samples and theta");
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < N; ++m) {
    if (!(theta[m] >= 0.0 && theta[m] < two_pi) || (m > 0 && !(theta[m] > theta[m - 1])))
      return set_error(AFD_ERR_INVALID, "theta must ascend strictly within [0, 2 pi) (index %d)", m);
    if (weights && !(weights[m] > 0.0 && weights[m] < 1e300))
      return set_error(AFD_ERR_INVALID, "weights must be positive and finite (index %d)", m);
  }
  if (!is_pow2(L) || L < (1 << NU_MIN_LOGN) || L > (1 << NU_MAX_LOGN))
    return set_error(AFD_ERR_INVALID, "L = %d: a power of two in [%d, %d]", L, 1 << NU_MIN_LOGN, 1 << NU_MAX_LOGN);
  AFD_TRY(check_radii(radii, M));
  AFD_TRY(resolve_device(o, dev));
  DeviceScope scope(dev);
  if (!scope.ok) return set_error(AFD_ERR_CUDA, "cannot make device %d current", dev);
  AFD_TRY(ensure_configured(dev));
  std::unique_ptr<afd_plan> p(new (std::nothrow) afd_plan());
  if (!p) return set_error(AFD_ERR_NOMEM, "host allocation failed");
  p->device = dev;
  p->opts = o;
  p->opts.persistent = 0;
  if (o.stream) {
    p->runner.main = static_cast<cudaStream_t>(o.stream);
  } else {
    CUDA_TRY(cudaStreamCreateWithFlags(&p->runner.main, cudaStreamNonBlocking));
    p->own_stream = true;
  }
  AFD_TRY(p->tables.build_nu(N, theta, weights, L, radii, M));
  *out = p.release();
  return AFD_OK;
}

afd_status afd_plan_destroy(afd_plan* plan) {
  if (!plan) return AFD_OK;
  DeviceScope scope(plan->device);
  if (plan->runner.main) cudaStreamSynchronize(plan->runner.main);
  delete plan;
  return AFD_OK;
}

afd_status afd_decompose_from(afd_plan* plan, const double* G, double E1_in, int K_max, double energy_tol,
                              double* a_out, double* coeff_out, double* delta_out, int* idx_out,
                              int* steps_done, double* G_final, double* E1_out) {
  clear_last_error();
  if (!plan || !G) return set_error(AFD_ERR_INVALID, "plan or G is NULL");
  if (!(E1_in >= 0.0) || std::isinf(E1_in)) return set_error(AFD_ERR_INVALID, "E1 must be finite and >= 0");
  if (K_max < 1 || K_max > (1 << 20)) return set_error(AFD_ERR_INVALID, "K_max = %d out of range", K_max);
  if (!(energy_tol >= 0.0)) return set_error(AFD_ERR_INVALID, "energy_tol must be >= 0");
  DeviceScope scope(plan->device);
  if (!scope.ok) return set_error(AFD_ERR_CUDA, "cannot make device %d current", plan->device);
  SlotPool& pool = plan->pool;
  cudaStream_t st = plan->runner.main;
  if (pool.n != 1 || pool.K_max != K_max) {
    CUDA_TRY(cudaStreamSynchronize(st));
    plan->runner.destroy();
    std::vector<const Tables*> t{&plan->tables};
    AFD_TRY(pool.build(t, K_max, plan->opts));
  }
  if (plan->own_stream) AFD_TRY(plan->runner.order_after_default());
  const bool stamps = plan->timer.on && pool.persistent && plan->opts.precision == AFD_FP32_GUARDED &&
                      !plan->tables.nu && is_pow2(plan->tables.N) && plan->tables.N <= (1 << PERSISTENT_MAX_LOGN);
  if (stamps && plan->phase_cap < K_max) {
    if (plan->phase_dev) cudaFree(plan->phase_dev);
    plan->phase_dev = nullptr;
    plan->phase_cap = 0;
    CUDA_TRY(cudaMalloc(&plan->phase_dev, sizeof(long long) * 8 * (size_t)K_max));
    plan->phase_cap = K_max;
  }
  pool.host[0].phase_clk = stamps ? plan->phase_dev : nullptr;
  pool.host[0].E1_given = E1_in;
  pool.host[0].force_a1_zero = (plan->opts.force_a1_zero && E1_in == 0.0) ? 1 : 0;
  AFD_TRY(pool.upload(energy_tol, st));
  CUDA_TRY(cudaMemcpyAsync(pool.G_dev, G, 16 * (size_t)plan->tables.samples(), cudaMemcpyDefault, st));
  AFD_TRY(plan->runner.run(pool, K_max, plan->opts.use_graph != 0, plan->cnt, &plan->timer));
  AFD_TRY(gather_device_outputs(pool, K_max, a_out, coeff_out, delta_out, idx_out, steps_done, E1_out, st));
  if (G_final)
    CUDA_TRY(cudaMemcpyAsync(G_final, pool.G_dev, 16 * (size_t)plan->tables.samples(), cudaMemcpyDefault, st));
  // (the pointers are classified while the device runs)
  double *a_h = host_or_null(a_out), *c_h = host_or_null(coeff_out), *d_h = host_or_null(delta_out);
  double* e1_h = host_or_null(E1_out);
  int *ix_h = host_or_null(idx_out), *sd_h = host_or_null(steps_done);
  AFD_TRY(fetch_results(pool, st, a_h || c_h || d_h || ix_h));
  const int steps = pool.ctl_host[0].k;
  plan->last_steps = steps;
  if (stamps && steps > 0) {
    std::vector<long long> c(8 * (size_t)steps);
    CUDA_TRY(cudaMemcpy(c.data(), plan->phase_dev, sizeof(long long) * c.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < steps; ++k)
      for (int i = 0; i < 7; ++i) plan->phase_sum[i] += (double)(c[8 * k + i + 1] - c[8 * k + i]);
    plan->phase_steps += steps;
  }
  if (a_h || c_h || d_h || ix_h) AFD_TRY(write_outputs(pool, 0, K_max, steps, a_h, c_h, d_h, ix_h));
  if (sd_h) *sd_h = steps;
  if (e1_h) *e1_h = pool.ctl_host[0].E1;
  if (pool.ctl_host[0].err & 4) return set_error(AFD_ERR_TIMEOUT, "a bounded wait on the device ran out at step %d", steps);
  if (pool.ctl_host[0].err & 2) return set_error(AFD_ERR_NUMERIC, "non-finite objective at step %d", steps);
  return AFD_OK;
}

afd_status afd_decompose(afd_plan* plan, const double* G, int K_max, double energy_tol, double* a_out,
                         double* coeff_out, double* delta_out, int* idx_out, int* steps_done) {
  return afd_decompose_from(plan, G, 0.0, K_max, energy_tol, a_out, coeff_out, delta_out, idx_out, steps_done,
                            nullptr, nullptr);
}

afd_status afd_plan_last_info(const afd_plan* plan, int* n_cand_out, int* flags_out, double* obj32_out) {
  if (!plan) return set_error(AFD_ERR_INVALID, "plan is NULL");
  if (!plan->pool.rec_fresh && plan->last_steps > 0) {
    DeviceScope scope(plan->device);
    if (!scope.ok) return set_error(AFD_ERR_CUDA, "cannot make device %d current", plan->device);
    AFD_TRY(fetch_records(const_cast<afd_plan*>(plan)->pool));  // the plan's last call has completed
  }
  const StepRec* r = plan->pool.rec_host;
  for (int k = 0; k < plan->last_steps && r; ++k) {
    if (n_cand_out) n_cand_out[k] = r[k].n_cand;
    if (flags_out) flags_out[k] = r[k].flags;
    if (obj32_out) obj32_out[k] = r[k].obj32;
  }
  return AFD_OK;
}

afd_status afd_plan_set_profiling(afd_plan* plan, int on) {
  if (!plan) return set_error(AFD_ERR_INVALID, "plan is NULL");
  plan->timer.on = on != 0;
  return AFD_OK;
}

afd_status afd_plan_counters(const afd_plan* plan, long long* kernel_launches, long long* grid_launches,
                             double* grid_ms) {
  if (!plan) return set_error(AFD_ERR_INVALID, "plan is NULL");
  if (kernel_launches) *kernel_launches = plan->cnt.launches;
  if (grid_launches) *grid_launches = plan->cnt.n[0];
  if (grid_ms) *grid_ms = plan->cnt.ms[0];
  return AFD_OK;
}

afd_status afd_plan_kernel_times(const afd_plan* plan, double* ms, long long* launches) {
  if (!plan) return set_error(AFD_ERR_INVALID, "plan is NULL");
  for (int i = 0; i < KINDS; ++i) {
    if (ms) ms[i] = plan->cnt.ms[i];
    if (launches) launches[i] = plan->cnt.n[i];
  }
  return AFD_OK;
}

afd_status afd_plan_phase_cycles(const afd_plan* plan, double* avg_cycles, long long* steps) {
  if (!plan) return set_error(AFD_ERR_INVALID, "plan is NULL");
  for (int i = 0; i < 7 && avg_cycles; ++i)
    avg_cycles[i] = plan->phase_steps ? plan->phase_sum[i] / (double)plan->phase_steps : 0.0;
  if (steps) *steps = plan->phase_steps;
  return AFD_OK;
}

afd_status afd_plan_get_stream(const afd_plan* plan, void** stream) {
  if (!plan || !stream) return set_error(AFD_ERR_INVALID, "plan or stream is NULL");
  *stream = plan->runner.main;
  return AFD_OK;
}

afd_status afd_plan_reset_counters(afd_plan* plan) {
  if (!plan) return set_error(AFD_ERR_INVALID, "plan is NULL");
  plan->cnt = Counters{};
  for (double& v : plan->phase_sum) v = 0.0;
  plan->phase_steps = 0;
  return AFD_OK;
}

// ----------------------------------------------------------------- batches --

afd_status afd_batch_create(afd_batch** out, int n_signals, const int* N, const double* radii, int M,
                            int K_max, const afd_plan_opts* opts) {
  clear_last_error();
  if (!out) return set_error(AFD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n_signals < 1 || !N) return set_error(AFD_ERR_INVALID, "need n_signals >= 1 and N");
  if (K_max < 1 || K_max > (1 << 20)) return set_error(AFD_ERR_INVALID, "K_max = %d out of range", K_max);
  afd_plan_opts o;
  int dev = 0;
  // every argument is checked before the first CUDA call
  AFD_TRY(resolve_opts(opts, o));
  if (o.offgrid_iters) return set_error(AFD_ERR_INVALID, "offgrid_iters: plans only");
  AFD_TRY(check_radii(radii, M));
  if (o.force_a1_zero && radii[0] != 0.0)
    return set_error(AFD_ERR_INVALID, "force_a1_zero needs radii[0] == 0");
  for (int i = 0; i < n_signals; ++i) AFD_TRY(check_size(N[i], o.precision, false, true));
  AFD_TRY(resolve_device(o, dev));
  DeviceScope scope(dev);
  if (!scope.ok) return set_error(AFD_ERR_CUDA, "cannot make device %d current", dev);
  AFD_TRY(ensure_configured(dev));
  std::unique_ptr<afd_batch> b(new (std::nothrow) afd_batch());
  if (!b) return set_error(AFD_ERR_NOMEM, "host allocation failed");
  b->device = dev;
  b->opts = o;
  b->N.assign(N, N + n_signals);
  if (o.stream) {
    b->runner.main = static_cast<cudaStream_t>(o.stream);
  } else {
    CUDA_TRY(cudaStreamCreateWithFlags(&b->runner.main, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  std::map<int, Tables*> by_n;
  std::vector<const Tables*> per_signal(n_signals);
  for (int i = 0; i < n_signals; ++i) {
    auto it = by_n.find(N[i]);
    if (it == by_n.end()) {
      b->tables.emplace_back(new Tables());
      AFD_TRY(b->tables.back()->build(N[i], radii, M, o.precision));
      it = by_n.emplace(N[i], b->tables.back().get()).first;
    }
    per_signal[i] = it->second;
  }
  // the single-signal persistent kernel is for plans; for a batch,
  // persistent = 2 picks the multi-signal kernel where it applies
  afd_plan_opts ob = o;
  ob.persistent = 0;
  AFD_TRY(b->pool.build(per_signal, K_max, ob, o.persistent == 2));
  *out = b.release();
  return AFD_OK;
}

afd_status afd_batch_run(afd_batch* b, const double* G_packed, double energy_tol, double* a_out,
                         double* coeff_out, double* delta_out, int* idx_out, int* steps_out) {
  clear_last_error();
  if (!b || !G_packed) return set_error(AFD_ERR_INVALID, "batch or G_packed is NULL");
  if (!(energy_tol >= 0.0)) return set_error(AFD_ERR_INVALID, "energy_tol must be >= 0");
  DeviceScope scope(b->device);
  if (!scope.ok) return set_error(AFD_ERR_CUDA, "cannot make device %d current", b->device);
  SlotPool& pool = b->pool;
  cudaStream_t st = b->runner.main;
  if (b->own_stream) AFD_TRY(b->runner.order_after_default());
  AFD_TRY(pool.upload(energy_tol, st));
  CUDA_TRY(cudaMemcpyAsync(pool.G_dev, G_packed, 8 * pool.g_total, cudaMemcpyDefault, st));
  if (!b->tuned && b->opts.autotune && b->opts.grid_variant < 0) {
    // before the first capture of the step sequence
    AFD_TRY(autotune(pool, b->device, st));
    b->runner.destroy_graph();
  }
  b->tuned = true;
  AFD_TRY(b->runner.run(pool, pool.K_max, b->opts.use_graph != 0, b->cnt, nullptr));
  AFD_TRY(gather_device_outputs(pool, pool.K_max, a_out, coeff_out, delta_out, idx_out, steps_out, nullptr, st));
  bool numeric = false, timeout = false;
  double *a_h = host_or_null(a_out), *c_h = host_or_null(coeff_out), *d_h = host_or_null(delta_out);
  int *ix_h = host_or_null(idx_out), *so_h = host_or_null(steps_out);
  const bool host_rec = a_h || c_h || d_h || ix_h;
  AFD_TRY(fetch_results(pool, st, host_rec));
  for (int i = 0; i < pool.n; ++i) {
    const int steps = pool.ctl_host[i].k;
    numeric |= (pool.ctl_host[i].err & 2) != 0;
    timeout |= (pool.ctl_host[i].err & 4) != 0;
    if (host_rec) AFD_TRY(write_outputs(pool, i, pool.K_max, steps, a_h, c_h, d_h, ix_h));
    if (so_h) so_h[i] = steps;
  }
  if (timeout) return set_error(AFD_ERR_TIMEOUT, "a bounded wait on the device ran out");
  if (numeric) return set_error(AFD_ERR_NUMERIC, "non-finite objective in at least one signal");
  return AFD_OK;
}

afd_status afd_batch_tuning(const afd_batch* b, int max_groups, int* n_groups, int* N_out, int* variant_out,
                            float* us_out) {
  if (!b) return set_error(AFD_ERR_INVALID, "batch is NULL");
  const auto& gs = b->pool.groups;
  if (n_groups) *n_groups = (int)gs.size();
  for (int i = 0; i < (int)gs.size() && i < max_groups; ++i) {
    if (N_out) N_out[i] = gs[i].N;
    if (variant_out) variant_out[i] = gs[i].variant;
    if (us_out) us_out[i] = gs[i].variant_us;
  }
  return AFD_OK;
}

afd_status afd_batch_counters(const afd_batch* b, long long* kernel_launches) {
  if (!b) return set_error(AFD_ERR_INVALID, "batch is NULL");
  if (kernel_launches) *kernel_launches = b->cnt.launches;
  return AFD_OK;
}

afd_status afd_batch_destroy(afd_batch* b) {
  if (!b) return AFD_OK;
  DeviceScope scope(b->device);
  if (b->runner.main) cudaStreamSynchronize(b->runner.main);
  delete b;
  return AFD_OK;
}

afd_status afd_decompose_batch(int n_signals, const int* N, const double* radii, int M,
                               const double* G_packed, int K_max, double energy_tol,
                               const afd_plan_opts* opts, double* a_out, double* coeff_out,
                               double* delta_out, int* idx_out, int* steps_out) {
  afd_batch* b = nullptr;
  AFD_TRY(afd_batch_create(&b, n_signals, N, radii, M, K_max, opts));
  afd_status s = afd_batch_run(b, G_packed, energy_tol, a_out, coeff_out, delta_out, idx_out, steps_out);
  afd_batch_destroy(b);
  return s;
}

}  // extern "C"
