// Internal structures shared by the CUDA kernels and the host runtime of the
// FFT-accelerated Core AFD library.  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>

namespace afd {

// Work split of the FP64 kernels (guard, update, energy): each CTA of
// FP64_THREADS threads owns FP64_CHUNK consecutive sample points, one per
// thread, so one signal's FP64 work spreads over N / 128 SMs.  GB300 issues
// FP64 at about 1/70 of its FP32 rate, so FP64 work is spread wide.  The split
// depends on N only, which keeps results identical alone and in a batch.
constexpr int FP64_THREADS = 128;
constexpr int FP64_CHUNK = 128;
constexpr int GUARD_PAR = 4;           // candidates in flight per guard launch
constexpr int MAX_LOGN_RESIDENT = 14;  // N <= 16384: one CTA holds one FFT
constexpr int TWO_PASS_LOGN = 16;      // N = 65536: two-pass FFT through HBM (FP32 plans only)
constexpr int MAX_LOGN = 16;           // largest power-of-two size of any path
// Longest transform one CTA holds on chip: 2^14 points in FP32, 2^13 in FP64.
inline __host__ __device__ constexpr int resident_logn(int prec) { return prec ? 14 : 13; }
// Transforms longer than that (FP32 N = 32768; FP64 N = 16384 .. 65536) are
// split by output index into 2^LS sub-transforms of the resident length: with
// S = 2^LS, NS = N / S and l = l' + p NS,
//   F(S j' + h) = sum_{l' < NS} [ w^{h l'} sum_{p < S} f(l' + p NS) exp(2 pi i h p / S) ] w_NS^{j' l'},
// one decimation-in-frequency step of radix S (the splitting of Theorem 2.1
// with radix S instead of 2).  Returns LS (0: not split).  FP32 N = 65536
// takes the two-pass path instead.
inline __host__ __device__ constexpr int split_log(int logN, int prec) {
  return (prec && logN == TWO_PASS_LOGN) ? 0 : (logN > resident_logn(prec) ? logN - resident_logn(prec) : 0);
}
constexpr int PERSISTENT_MAX_LOGN = 12;  // persistent single-signal kernel up to N = 4096
constexpr int MIN_LOGN = 3;            // N >= 8
constexpr int MAX_CAP = 64;            // guard candidates per step, upper bound

inline __host__ __device__ int chunks_of(int N) { return (N + FP64_CHUNK - 1) / FP64_CHUNK; }
// (x mod N) for x in (-N, 2N); N need not be a power of two
inline __host__ __device__ int wrap_mod(int x, int N) { return x < 0 ? x + N : (x >= N ? x - N : x); }
constexpr int MIXED_MAX_PASSES = 24;
constexpr int RF_MAX_CTAS = 64;  // CTAs of the off-grid refinement of one signal
// Grid-barrier counter of the persistent kernels, their error word and the
// multi-signal kernel's work-item ticket: a 128-byte line each, zeroed before
// a launch.
constexpr int BAR_BYTES = 384;
// Largest shared-memory footprint (two ping-pong buffers of N points) of the
// mixed-radix kernels: N <= 12800 in FP32, N <= 6400 in FP64.
constexpr int MIXED_MAX_SMEM = 204800;

// Radix schedule of the mixed-radix Stockham transform of length
// N = 2^a 3^b 5^c 7^d 11^e 13^f: radix-16 passes, one pass of 8, 4 or 2 for
// the rest of the power of two, then one pass per odd prime factor (3, 5, 7,
// 11, 13, in that order).  Returns the number of passes written to radix[],
// or -1 if N has another prime factor or needs more than MIXED_MAX_PASSES
// passes.
template <typename I>
inline __host__ __device__ int mixed_schedule(int N, I* radix) {
  if (N < 2) return -1;
  int n = N, np = 0;
  while (n % 16 == 0 && np < MIXED_MAX_PASSES) { radix[np++] = 16; n /= 16; }
  if (n % 8 == 0 && np < MIXED_MAX_PASSES) { radix[np++] = 8; n /= 8; }
  else if (n % 4 == 0 && np < MIXED_MAX_PASSES) { radix[np++] = 4; n /= 4; }
  else if (n % 2 == 0 && np < MIXED_MAX_PASSES) { radix[np++] = 2; n /= 2; }
  for (int p = 3; p <= 13; p += 2) {  // 3, 5, 7, 9 (never divides: 3 is gone), 11, 13
    while (n % p == 0 && np < MIXED_MAX_PASSES) { radix[np++] = (I)p; n /= p; }
  }
  return n == 1 ? np : -1;
}

// Per (N, radii) tables, owned by a plan, read-only in kernels.
struct PlanDev {
  int N, logN, M, B;        // B = FftSchedule::pow_b(logN - ls); the high power table has N / B entries
  const double* radii;      // [M] ascending radii r_s in [0, 1)
  const double2* tw64;      // [N] exp(+2 pi i k / N) in FP64 (also the sample points z_m)
  const float2* st32;       // [FftSchedule::tw_size] FFT stage twiddles, FP32
  const float4* st32p;      // [tw_size / 2] the same, pairs of entries (2j, 2j+1) as
                            // (re_2j, re_2j+1, im_2j, im_2j+1) for the paired FP32 transforms
  const double2* st64;      // the same in FP64
  const float* rlo32;       // [M * B]        r_s^q,        q = 0..B-1
  const float* rhi32;       // [M * (N / B)]  r_s^(B h),    h = 0..N/B-1
  const double* rlo64;
  const double* rhi64;
  const float* wsq32;       // [M] w_s^2 with w_s = sqrt(1 - r_s^2) / (1 - r_s^N)
  const double* w64;        // [M] w_s
  const double* sq64;       // [M] sqrt(1 - r_s^2)
  const double* rho64;      // [M] 1 / ||e_a||_N^2 = (1 - r_s^N) / (1 + r_s^N) (renormalised selection)
  const float* rho32;       // [M] the same in FP32
  const double2* K64;       // [M * N] 1 / (1 - r_s exp(2 pi i d / N)), FP64
  const float2* tw32n;      // [N] exp(+2 pi i k / N) in FP32 (two-pass, mixed-radix); two-pass:
                            // followed by [4096] exp(+2 pi i m / 4096)
  double inv_n;             // 1 / N (exact for powers of two)
  // Non-uniform samples (nN > 0): the grid has N angles; the signal is known
  // at exp(i theta_m), m < nN, with quadrature weights w_m (sum 1)
  int nN;                   // number of samples (0: the N equispaced samples)
  int nLc;                  // length of the non-uniform DFT: the most folds of any radius x N
  const double2* nz64;      // [nN] exp(i theta_m)
  const double* nw64;       // [nN] w_m
  const unsigned long long* nU;  // [nN] theta_m / 2 pi as a 64-bit fixed-point fraction
  const int* nP;            // [M] folds of radius s: r_s^(nP N) <= 2^-64
  const float* nrN32;       // [M] r_s^N in FP32
  int mix_npass;            // mixed-radix path (N not a power of two): passes and radices
  unsigned char mix_radix[MIXED_MAX_PASSES];
  int ls;                   // split_log(logN, precision): 2^ls sub-transforms per radius (0: none)
};

// One greedy step's outcome, written on the device.
struct StepRec {
  int s, j;                 // selected grid index (radius s, angle j)
  int n_cand;               // FP64 guard candidates evaluated (FP32 path)
  int flags;                // bit 0: more points in the guard window than the cap; bit 1: non-finite
                            // objective; bit 2: a bounded wait ran out
  double a_re, a_im;        // a_k = r_s exp(2 pi i j / N)
  double c_re, c_im;        // <G_k, e_{a_k}>~
  double obj;               // |c|^2
  double energy;            // E_{k+1} = (1/N) sum |G_{k+1}|^2
  double delta;             // E_{k+1} / E_1
  double obj32;             // largest FP32 objective of the step (FP32 path)
};

// Mutable per-signal control block.
struct SlotCtl {
  int k;                    // greedy steps completed
  int done;                 // set once the stop rule fires
  int n_cand;               // candidates of the current step
  int err;                  // sticky error bits (StepRec::flags)
  double E1;                // initial energy
  unsigned cnt_grid, cnt_guard, cnt_update;  // last-CTA counters
  unsigned vmax_bits;       // FP32 path: bits of the step's largest objective (atomicMax)
  unsigned bar_count, bar_gen;  // bar_gen: grid barriers the off-grid refinement has passed
  unsigned vmax2[2];        // persistent kernel: vmax_bits of even / odd steps
  double Estart;            // energy of the remainder the call started from
};

struct Top2F { float v1, v2; int j1, j2; };
struct Top2D { double v1, v2; int j1, j2; double2 f1, f2; };

// Everything a kernel needs about one signal in flight.
struct SlotDev {
  PlanDev p;
  int K_max;
  int prec;                 // 0: FP64 plain, 1: FP32 grid + FP64 guard
  int cap;                  // guard candidate cap
  int force_a1_zero;
  int renorm;               // select by the objective times rho (renormalised)
  double tol;               // stop once delta <= tol (0: never)
  double tau;               // guard window: obj32 >= (1 - tau) * max32
  double E1_given;          // > 0: reference energy E_1 of a resumed decomposition
  double2* G;               // [N] remainder G_k(z_m), FP64
  double2* G2;              // persistent kernel: second remainder buffer (odd steps)
  float2* g32b;             // persistent kernel: second FP32 copy (odd steps)
  float2* g32;              // [N] G_k(z_m) / N rounded to FP32 (input of the FP32 forward FFT)
  float2* c32;              // [N] spectrum c_l / N, FP32
  float2* X;                // two-pass path: [M * N] pass-1 output, X_s[j2][l1]
  double2* c64;             // [N] spectrum c_l / N, FP64
  void* top2;               // [M] Top2F or Top2D
  int2* cand;               // [cap] (s, j)
  double2* gpart;           // [cap * chunks_of(N)] guard partial sums (x4: persistent, per warp)
  double* epart;            // [chunks_of(N)] energy partial sums (persistent: x4 per warp, x K_max steps)
  double* rfpart;           // off-grid refinement: [2][RF_MAX_CTAS][6] per-CTA sums of a Newton pass
  StepRec* rec;             // [K_max]
  SlotCtl* ctl;
  long long* phase_clk;     // persistent kernel, optional: 8 SM-clock stamps per step (CTA 0)
  unsigned* bar;            // persistent kernel: grid-barrier arrival counter (own 128-byte line)
};
// Selection weight of radius s: the FP32 objective weight w_s^2 and the FP64
// factor applied to |c|^2, both times rho_s when the selection is renormalised.
__device__ __forceinline__ float obj_w32(const SlotDev& sd, int s) {
  const float w = sd.p.wsq32[s];
  return sd.renorm ? w * sd.p.rho32[s] : w;
}
__device__ __forceinline__ double obj_rho64(const SlotDev& sd, int s) { return sd.renorm ? sd.p.rho64[s] : 1.0; }

// Host-visible layout sizes (the bench reports per-step transfer bytes from them).
static_assert(sizeof(StepRec) == 80, "StepRec layout");
static_assert(sizeof(SlotCtl) == 64, "SlotCtl layout");
static_assert(sizeof(SlotDev) == 408, "SlotDev layout");

// The multi-signal persistent kernel (afd_multi.cu): one N-class of signals
// (ids[first .. first + count)) and its work split.
constexpr int MULTI_THREADS = 512;
constexpr int MULTI_MAX_CLASSES = 16;
struct MultiClass {
  int logN, first, count, Mmax;  // logN < 0: a mixed-radix size N (256-thread build only)
  int N;
  int tiles;    // grid items (radius tiles) per signal
  int gpar;     // guard: candidates in flight per signal (as launch_guard)
  int fgroups;  // forward: signals per CTA (transform groups)
};
struct MultiArgs {
  const SlotDev* slots;
  const int* ids;        // the signals of the steps, grouped by class
  const int* fresh_ids;  // the signals to initialise first, grouped by class
  unsigned* bar;         // BAR_BYTES, zeroed before the launch: barrier counter, error word, ticket
  int K;                 // greedy steps
  int final_forward;     // 1: transform the remainder after the last step too (serving)
  int n_cls, n_fresh;
  MultiClass cls[MULTI_MAX_CLASSES], fresh[MULTI_MAX_CLASSES];
};
bool multi_size_ok(int logN);  // FP32 powers of two 8 .. 16384
void multi_class_shape(int logN, int Mmax, int count, int cap, MultiClass* c);  // all but first
// the same for a mixed-radix size N (FP32 path): one radius per grid item
void multi_class_shape_mixed(int N, int Mmax, int count, int cap, MultiClass* c);
cudaError_t multi_configure();
// One cooperative launch: the fresh signals' initialisation, then K steps.
cudaError_t launch_multi(const MultiArgs& a, cudaStream_t st);

// Kernel launchers (afd_kernels.cu).  `ids` lists the slots of one launch, all
// with the same logN; `n` is their number.  Each returns the launch status.
cudaError_t launch_init(const SlotDev* slots, const int* ids, int n, int N, cudaStream_t st);
cudaError_t launch_grid(const SlotDev* slots, const int* ids, int n, int logN, int prec, int Mmax,
                        cudaStream_t st, int variant = 0);
// Grid-kernel variants (0: default; 1: 32 points per thread; 2: 512-thread
// CTAs), all bitwise equivalent; which exist for (logN, precision).
constexpr int GRID_VARIANTS = 3;
bool grid_variant_ok(int logN, int prec, int variant);
// Whole FP32-path decomposition of slot 0 in one cooperative launch (after
// launch_init); logN <= MAX_LOGN_RESIDENT.
cudaError_t launch_persistent(const SlotDev* slots, int logN, int M, cudaStream_t st);
// Self-tests of the bounded waits: one CTA whose wait can never be satisfied
// (the persistent kernel's grid barrier; an mbarrier of the TMA-staged
// passes); elapsed_ns gets the wait's duration by the GPU's global timer.
cudaError_t launch_selftest_barrier(const SlotDev* slot, unsigned long long* elapsed_ns, cudaStream_t st);
cudaError_t launch_selftest_mbarrier(SlotCtl* ctl, unsigned long long* elapsed_ns, cudaStream_t st);
cudaError_t launch_guard(const SlotDev* slots, const int* ids, int n, int N, int cap, cudaStream_t st);
cudaError_t launch_update(const SlotDev* slots, const int* ids, int n, int N, cudaStream_t st);
// Off-grid refinement of each signal's step winner (afd_offgrid.cu), then the
// update at the refined point.
cudaError_t launch_refine(const SlotDev* slots, const int* ids, int n, int N, int iters, cudaStream_t st);
cudaError_t launch_update_offgrid(const SlotDev* slots, const int* ids, int n, int N, cudaStream_t st);
// Mixed-radix path (afd_mixed.cu): N = 2^a 3^b 5^c, not a power of two.
cudaError_t launch_grid_mixed(const SlotDev* slots, const int* ids, int n, int N, int prec, int Mmax,
                              cudaStream_t st);
cudaError_t launch_forward_mixed(const SlotDev* slots, const int* ids, int n, int N, int prec, cudaStream_t st);
cudaError_t mixed_configure();
// Non-uniform samples (afd_nu.cu), single-signal FP32-path plans.
constexpr int NU_MIN_LOGN = 3, NU_MAX_LOGN = 13, NU_MAX_FOLDS = 64;
cudaError_t launch_nudft(const SlotDev* slots, const int* ids, int Lc, cudaStream_t st);
cudaError_t launch_grid_nu(const SlotDev* slots, const int* ids, int logN, int M, cudaStream_t st);
cudaError_t launch_guard_nu(const SlotDev* slots, const int* ids, int nN, int cap, cudaStream_t st);
cudaError_t launch_update_nu(const SlotDev* slots, const int* ids, int nN, bool init, cudaStream_t st);
cudaError_t nu_configure();
size_t mixed_smem_bytes(int N, int prec);
cudaError_t launch_forward(const SlotDev* slots, const int* ids, int n, int logN, int prec,
                           cudaStream_t st);
// Step records of signals 0..n-1 into caller device arrays on stream st (any
// pointer may be NULL; the layout of afd_batch_run with K_stride steps per
// signal); steps_out[i] and E1_out (signal 0) from the control blocks.
cudaError_t launch_gather(const StepRec* rec, const SlotCtl* ctl, int n, int K_max, int K_stride, double* a,
                          double* coeff, double* delta, int* idx, int* steps_out, double* E1_out, cudaStream_t st);
// Fills K[s * N + d] = 1 / (1 - r_s exp(2 pi i d / N)) for a plan.
cudaError_t launch_kernel_table(const double* radii, int M, int N, double2* K, cudaStream_t st);
// Shared memory (bytes) the grid kernel needs for this logN and precision.
size_t grid_smem_bytes(int logN, int prec);
size_t forward_smem_bytes(int logN, int prec);
int grid_ffts_per_cta(int logN, int prec);
cudaError_t configure_kernels();
// Sets the text afd_last_error() returns on the calling thread.
void set_last_error_text(const char* text);

}  // namespace afd
