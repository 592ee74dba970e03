// Serving loop for Core AFD decompositions: continuous batching.
//
// Requests (one signal each, with its own N, radii, step limit and energy
// tolerance) arrive through afd_serve_submit from any host thread.  A worker
// thread owns the device side:
//   admit   queued requests, oldest first, into free slots while the device
//           memory budget allows (slot memory from a size-class arena, plan
//           tables from a cache; both count against the budget);
//   tick    one greedy step for every active slot: per size class N the
//           initialisation of newly admitted slots, then grid, guard, update
//           and forward kernels over all of that class's slots;
//   retire  slots whose stop rule fired (delta <= tol or K steps): their step
//           records are copied to the host, the request completes and the
//           slot and its memory are reused by the next admission.
//   evict   slots whose request was suspended (afd_serve_suspend): the
//           remainder G_k, the step records and E_1 go to host memory and the
//           slot is freed; afd_serve_resume queues the request again, and its
//           admission restores that state (the initialisation recomputes the
//           FP32 copy and the spectrum from G_k, with E_1 given), so the
//           decomposition continues bit-identically.
// Requests that arrive while others run join at the next tick, so their work
// overlaps on the device.  A request computes exactly what afd_decompose
// computes for it alone: the kernels, their work split (which depends on N
// only) and the plan tables are the same.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/afd.h"
#include "afd_host.h"
#include "afd_internal.h"

using namespace afd;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlots = 4096;
// Greedy steps of every active request per multi-signal launch: the host's
// per-tick work (the launch, the control-block read, admission and
// retirement) is paid once per this many steps; a request stops on the
// device at its own last step, and arrivals wait at most one tick.
constexpr int kStepsPerTick = 4;

// Device arena: power-of-two size classes (>= 64 KiB) carved from 64 MiB
// chunks, or a dedicated allocation for larger blocks.  Every byte obtained
// from cudaMalloc counts against the budget; freed blocks go to their class's
// free list.
class Arena {
 public:
  static constexpr size_t kMin = size_t(64) << 10;
  // chunk size: a power of two near budget / 16, between 1 MiB and 64 MiB
  explicit Arena(size_t budget) : budget_(budget) {
    kChunk = size_t(1) << 20;
    while (kChunk < (size_t(64) << 20) && 2 * kChunk <= budget / 16) kChunk <<= 1;
  }
  ~Arena() {
    for (void* c : chunks_) cudaFree(c);
  }
  static size_t class_size(size_t bytes) {
    size_t c = kMin;
    while (c < bytes) c <<= 1;
    return c;
  }
  // AFD_ERR_BUDGET when the budget does not allow it now.
  afd_status alloc(size_t bytes, void** out) {
    const size_t c = class_size(bytes);
    auto& fl = free_[c];
    if (!fl.empty()) {
      *out = fl.back();
      fl.pop_back();
      in_use_ += c;
      return AFD_OK;
    }
    if (c >= kChunk) {
      if (reserved_ + c > budget_) return AFD_ERR_BUDGET;
      void* p = nullptr;
      CUDA_TRY(cudaMalloc(&p, c));
      chunks_.push_back(p);
      chunk_bytes_.push_back(c);
      reserved_ += c;
      in_use_ += c;
      *out = p;
      return AFD_OK;
    }
    if (!bump_ || bump_left_ < c) {
      if (reserved_ + kChunk > budget_) return AFD_ERR_BUDGET;
      void* p = nullptr;
      CUDA_TRY(cudaMalloc(&p, kChunk));
      chunks_.push_back(p);
      chunk_bytes_.push_back(kChunk);
      reserved_ += kChunk;
      bump_ = static_cast<char*>(p);
      bump_left_ = kChunk;
    }
    *out = bump_;
    bump_ += c;
    bump_left_ -= c;
    in_use_ += c;
    return AFD_OK;
  }
  void release(void* p, size_t bytes) {
    const size_t c = class_size(bytes);
    free_[c].push_back(p);
    in_use_ -= c;
  }
  // Memory allocated elsewhere (plan tables) that counts against the budget.
  bool charge(size_t bytes) {
    if (reserved_ + bytes > budget_) return false;
    reserved_ += bytes;
    return true;
  }
  void uncharge(size_t bytes) { reserved_ -= bytes; }
  // Returns every chunk to the driver; only valid when no block is in use.
  void reset() {
    for (void* c : chunks_) cudaFree(c);
    for (auto& kv : chunk_bytes_) reserved_ -= kv;
    chunks_.clear();
    chunk_bytes_.clear();
    free_.clear();
    bump_ = nullptr;
    bump_left_ = 0;
  }
  size_t budget() const { return budget_; }
  size_t reserved() const { return reserved_; }
  size_t in_use() const { return in_use_; }

 private:
  size_t kChunk;
  size_t budget_, reserved_ = 0, in_use_ = 0;
  std::vector<void*> chunks_;
  std::vector<size_t> chunk_bytes_;
  std::map<size_t, std::vector<void*>> free_;
  char* bump_ = nullptr;
  size_t bump_left_ = 0;
};

struct SlotLayout {
  size_t G, g32, c, top2, cand, gpart, epart, rec, total;
};

SlotLayout slot_layout(int N, int M, int K, int prec, int cap) {
  SlotLayout L{};
  size_t off = 0;
  auto place = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
  L.G = place(16 * (size_t)N);
  L.g32 = place(prec ? 8 * (size_t)N : 0);
  L.c = place((prec ? 8 : 16) * (size_t)N);
  // one best pair per radius, or per sub-transform of a split size
  L.top2 = place((prec ? sizeof(Top2F) : sizeof(Top2D)) * ((size_t)M << split_log(ilog2(N), prec)));
  L.cand = place(sizeof(int2) * cap);
  L.gpart = place(sizeof(double2) * cap * (size_t)chunks_of(N));
  L.epart = place(sizeof(double) * (size_t)chunks_of(N));
  L.rec = place(sizeof(StepRec) * (size_t)K);
  L.total = off;
  return L;
}

struct Request {
  uint64_t id = 0;
  int N = 0, K = 0;
  double tol = 0.0;
  std::vector<double> radii, G;  // G: the samples to start from (G_k after a suspension)
  int state = 0;  // 0 queued, 1 active, 2 done, 3 suspended
  bool suspend = false;  // asked to leave its slot at the next tick boundary
  afd_status status = AFD_OK;
  int steps = 0;              // steps done (records in recs)
  double E1 = 0.0;            // E_1 of a suspended decomposition (0: not started)
  std::vector<StepRec> recs;
  Clock::time_point t_submit, t_done;
};

struct Slot {
  bool used = false;
  bool fresh = false;
  uint64_t req = 0;
  void* block = nullptr;
  size_t bytes = 0;
  const Tables* tables = nullptr;
  int logN = 0, K = 0;
  SlotLayout L{};
};

}  // namespace

struct afd_server {
  int device = 0;
  afd_plan_opts opts{};
  bool own_stream = false;
  cudaStream_t stream = nullptr;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_id = 1;
  std::map<std::vector<double>, std::unique_ptr<Tables>> plans;  // key: N, radii...
  std::vector<Slot> slots;
  int n_active = 0;
  SlotDev* slots_dev = nullptr;
  SlotCtl* ctl_dev = nullptr;
  int* ids_dev = nullptr;
  unsigned* bar_dev = nullptr;      // the multi-signal kernel's barrier counter and error word
  SlotDev* slotdev_host = nullptr;  // pinned
  SlotCtl* ctl_host = nullptr;      // pinned
  int* ids_host = nullptr;          // pinned
  StepRec* rec_stage = nullptr;     // pinned
  size_t rec_stage_cap = 0;
  std::thread worker;
  bool stop = false;
  afd_status fatal = AFD_OK;
  std::string fatal_text;
  afd_serve_stats st{};
  size_t fixed_bytes = 0;

  explicit afd_server(size_t budget) : arena(budget) {}
  ~afd_server() {
    if (slots_dev) cudaFree(slots_dev);
    if (ctl_dev) cudaFree(ctl_dev);
    if (ids_dev) cudaFree(ids_dev);
    if (bar_dev) cudaFree(bar_dev);
    if (slotdev_host) cudaFreeHost(slotdev_host);
    if (ctl_host) cudaFreeHost(ctl_host);
    if (ids_host) cudaFreeHost(ids_host);
    if (rec_stage) cudaFreeHost(rec_stage);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  // ---------------------------------------------------------- worker side --

  // Plan tables for (N, radii): cached; creation charges the budget.
  afd_status tables_for(const Request& r, const Tables** out) {
    std::vector<double> key;
    key.reserve(r.radii.size() + 1);
    key.push_back((double)r.N);
    key.insert(key.end(), r.radii.begin(), r.radii.end());
    auto it = plans.find(key);
    if (it != plans.end()) {
      *out = it->second.get();
      return AFD_OK;
    }
    std::unique_ptr<Tables> t(new (std::nothrow) Tables());
    if (!t) return AFD_ERR_NOMEM;
    AFD_TRY(t->build(r.N, r.radii.data(), (int)r.radii.size(), opts.precision));
    if (!arena.charge(t->bytes)) return AFD_ERR_BUDGET;
    *out = t.get();
    plans.emplace(std::move(key), std::move(t));
    return AFD_OK;
  }

  // Moves queued requests into free slots while slots and memory allow.
  // Called with mu held.
  afd_status admit() {
    while (!queue.empty()) {
      Request& r = *reqs[queue.front()];
      int si = -1;
      for (int i = 0; i < kMaxSlots; ++i)
        if (!slots[i].used) { si = i; break; }
      if (si < 0) return AFD_OK;
      const Tables* t = nullptr;
      afd_status s = tables_for(r, &t);
      if (s == AFD_ERR_BUDGET) return AFD_OK;  // wait for memory
      if (s != AFD_OK) return s;
      const int prec = opts.precision, cap = prec == AFD_FP32_GUARDED ? opts.guard_cap : 1;
      const SlotLayout L = slot_layout(r.N, (int)r.radii.size(), r.K, prec, cap);
      void* block = nullptr;
      s = arena.alloc(L.total, &block);
      if (s == AFD_ERR_BUDGET) return AFD_OK;  // wait for a retirement
      if (s != AFD_OK) return s;
      char* b = static_cast<char*>(block);
      SlotDev d{};
      d.p = t->dev;
      d.K_max = r.K;
      d.prec = prec;
      d.cap = cap;
      d.force_a1_zero = opts.force_a1_zero;
      d.renorm = opts.renormalise != 0;
      d.tol = r.tol;
      d.tau = opts.guard_tau;
      d.E1_given = r.E1;  // > 0 when resuming
      d.G = reinterpret_cast<double2*>(b + L.G);
      d.g32 = prec ? reinterpret_cast<float2*>(b + L.g32) : nullptr;
      d.c32 = prec ? reinterpret_cast<float2*>(b + L.c) : nullptr;
      d.c64 = prec ? nullptr : reinterpret_cast<double2*>(b + L.c);
      d.top2 = b + L.top2;
      d.cand = reinterpret_cast<int2*>(b + L.cand);
      d.gpart = reinterpret_cast<double2*>(b + L.gpart);
      d.epart = reinterpret_cast<double*>(b + L.epart);
      d.rec = reinterpret_cast<StepRec*>(b + L.rec);
      d.ctl = ctl_dev + si;
      slotdev_host[si] = d;
      CUDA_TRY(cudaMemcpyAsync(slots_dev + si, slotdev_host + si, sizeof(SlotDev), cudaMemcpyHostToDevice,
                               stream));
      CUDA_TRY(cudaMemcpyAsync(d.G, r.G.data(), 16 * (size_t)r.N, cudaMemcpyHostToDevice, stream));
      // control block: zero, or the step count of a resumed decomposition
      // (its records go back to the slot)
      ctl_host[si] = SlotCtl{};
      ctl_host[si].k = r.steps;
      CUDA_TRY(cudaMemcpyAsync(ctl_dev + si, ctl_host + si, sizeof(SlotCtl), cudaMemcpyHostToDevice, stream));
      if (r.steps > 0)
        CUDA_TRY(cudaMemcpyAsync(d.rec, r.recs.data(), sizeof(StepRec) * (size_t)r.steps, cudaMemcpyHostToDevice,
                                 stream));
      Slot& sl = slots[si];
      sl.used = true;
      sl.fresh = true;
      sl.req = r.id;
      sl.block = block;
      sl.bytes = L.total;
      sl.tables = t;
      sl.logN = ilog2(r.N);
      sl.K = r.K;
      sl.L = L;
      r.state = 1;
      r.G.clear();
      r.G.shrink_to_fit();
      queue.pop_front();
      ++n_active;
    }
    return AFD_OK;
  }

  // One greedy step for every active slot.  Worker thread only.
  afd_status tick() {
    std::vector<int> fresh[MAX_LOGN + 1], all[MAX_LOGN + 1];
    int Mmax[MAX_LOGN + 1] = {};
    int hi = 0;
    for (int i = 0; i < kMaxSlots; ++i) {
      const Slot& s = slots[i];
      if (!s.used) continue;
      hi = i + 1;
      all[s.logN].push_back(i);
      if (s.fresh) fresh[s.logN].push_back(i);
      Mmax[s.logN] = std::max(Mmax[s.logN], s.tables->M);
    }
    size_t n_ids = 0;
    size_t off_fresh[MAX_LOGN + 1], off_all[MAX_LOGN + 1];
    for (int l = 0; l <= MAX_LOGN; ++l) {
      off_fresh[l] = n_ids;
      for (int i : fresh[l]) ids_host[n_ids++] = i;
      off_all[l] = n_ids;
      for (int i : all[l]) ids_host[n_ids++] = i;
    }
    CUDA_TRY(cudaMemcpyAsync(ids_dev, ids_host, sizeof(int) * n_ids, cudaMemcpyHostToDevice, stream));
    const int prec = opts.precision;
    long long launches = 0;
    // FP32 path with every active size on chip: the whole tick (the fresh
    // requests' initialisation, then kStepsPerTick steps of every request)
    // is one multi-signal persistent launch
    bool multi = prec == AFD_FP32_GUARDED && opts.persistent != 0;
    for (int l = 0; l <= MAX_LOGN; ++l) multi = multi && (all[l].empty() || multi_size_ok(l));
    if (multi) {
      MultiArgs a{};
      a.slots = slots_dev;
      a.ids = ids_dev;
      a.fresh_ids = ids_dev;
      a.bar = bar_dev;
      a.K = kStepsPerTick;
      a.final_forward = 1;
      for (int l = 0; l <= MAX_LOGN; ++l) {
        if (!all[l].empty()) {
          MultiClass& c = a.cls[a.n_cls++];
          multi_class_shape(l, Mmax[l], (int)all[l].size(), opts.guard_cap, &c);
          c.first = (int)off_all[l];
        }
        if (!fresh[l].empty()) {
          MultiClass& f = a.fresh[a.n_fresh++];
          multi_class_shape(l, Mmax[l], (int)fresh[l].size(), opts.guard_cap, &f);
          f.first = (int)off_fresh[l];
        }
      }
      CUDA_TRY(cudaMemsetAsync(bar_dev, 0, BAR_BYTES, stream));
      CUDA_TRY(launch_multi(a, stream));
      launches = 1;
    }
    for (int l = 0; !multi && l <= MAX_LOGN; ++l) {
      if (all[l].empty()) continue;
      const int nf = (int)fresh[l].size(), na = (int)all[l].size();
      if (nf) {
        CUDA_TRY(launch_init(slots_dev, ids_dev + off_fresh[l], nf, 1 << l, stream));
        CUDA_TRY(launch_forward(slots_dev, ids_dev + off_fresh[l], nf, l, prec, stream));
        launches += 2;
      }
      const int* ids = ids_dev + off_all[l];
      CUDA_TRY(launch_grid(slots_dev, ids, na, l, prec, Mmax[l], stream));
      if (prec == AFD_FP32_GUARDED) {
        CUDA_TRY(launch_guard(slots_dev, ids, na, 1 << l, opts.guard_cap, stream));
        ++launches;
      }
      CUDA_TRY(launch_update(slots_dev, ids, na, 1 << l, stream));
      CUDA_TRY(launch_forward(slots_dev, ids, na, l, prec, stream));
      launches += 3;
    }
    CUDA_TRY(cudaMemcpyAsync(ctl_host, ctl_dev, sizeof(SlotCtl) * hi, cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    for (int i = 0; i < hi; ++i) slots[i].fresh = false;
    std::lock_guard<std::mutex> lk(mu);
    st.ticks += 1;
    st.kernel_launches += launches;
    return AFD_OK;
  }

  // Moves the slots of suspended requests to host memory (after retire: a
  // request that finished in the last tick completes instead).
  afd_status evict() {
    std::vector<int> out;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (int i = 0; i < kMaxSlots; ++i) {
        if (!slots[i].used) continue;
        auto it = reqs.find(slots[i].req);
        if (it != reqs.end() && it->second->suspend) out.push_back(i);
      }
    }
    if (out.empty()) return AFD_OK;
    std::vector<std::vector<double>> G(out.size());
    std::vector<std::vector<StepRec>> R(out.size());
    for (size_t q = 0; q < out.size(); ++q) {
      const int i = out[q];
      const Slot& sl = slots[i];
      const int k = ctl_host[i].k;
      const int N = slotdev_host[i].p.N;
      G[q].resize(2 * (size_t)N);
      R[q].resize((size_t)k);
      CUDA_TRY(cudaMemcpyAsync(G[q].data(), slotdev_host[i].G, 16 * (size_t)N, cudaMemcpyDeviceToHost, stream));
      if (k > 0)
        CUDA_TRY(cudaMemcpyAsync(R[q].data(), static_cast<char*>(sl.block) + sl.L.rec, sizeof(StepRec) * k,
                                 cudaMemcpyDeviceToHost, stream));
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    std::lock_guard<std::mutex> lk(mu);
    for (size_t q = 0; q < out.size(); ++q) {
      const int i = out[q];
      Slot& sl = slots[i];
      auto it = reqs.find(sl.req);
      if (it != reqs.end()) {
        Request& r = *it->second;
        r.G = std::move(G[q]);
        r.recs = std::move(R[q]);
        r.steps = ctl_host[i].k;
        r.E1 = ctl_host[i].E1;
        r.state = 3;
        r.suspend = false;
        st.suspended += 1;
      }
      arena.release(sl.block, sl.bytes);
      sl = Slot{};
      --n_active;
    }
    cv_done.notify_all();
    return AFD_OK;
  }

  // Copies the records of finished slots to their requests and frees them.
  afd_status retire() {
    std::vector<int> done;
    size_t need = 0;
    for (int i = 0; i < kMaxSlots; ++i) {
      // (a bounded wait that ran out also ends the request)
      if (slots[i].used && (ctl_host[i].done || (ctl_host[i].err & 4))) {
        done.push_back(i);
        need += (size_t)ctl_host[i].k;
      }
    }
    if (done.empty()) return AFD_OK;
    if (need > rec_stage_cap) {
      if (rec_stage) cudaFreeHost(rec_stage);
      rec_stage = nullptr;
      rec_stage_cap = 0;
      CUDA_TRY(cudaMallocHost((void**)&rec_stage, sizeof(StepRec) * std::max<size_t>(need, 1024)));
      rec_stage_cap = std::max<size_t>(need, 1024);
    }
    size_t off = 0;
    for (int i : done) {
      const int k = ctl_host[i].k;
      if (k > 0)
        CUDA_TRY(cudaMemcpyAsync(rec_stage + off, static_cast<char*>(slots[i].block) + slots[i].L.rec,
                                 sizeof(StepRec) * k, cudaMemcpyDeviceToHost, stream));
      off += k;
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    std::lock_guard<std::mutex> lk(mu);
    off = 0;
    const auto now = Clock::now();
    for (int i : done) {
      Slot& sl = slots[i];
      const int k = ctl_host[i].k;
      auto it = reqs.find(sl.req);
      if (it != reqs.end()) {
        Request& r = *it->second;
        r.recs.assign(rec_stage + off, rec_stage + off + k);
        r.steps = k;
        r.status = (ctl_host[i].err & 4) ? AFD_ERR_TIMEOUT : ((ctl_host[i].err & 2) ? AFD_ERR_NUMERIC : AFD_OK);
        r.state = 2;
        r.t_done = now;
        st.completed += 1;
      }
      off += k;
      arena.release(sl.block, sl.bytes);
      sl = Slot{};
      --n_active;
    }
    cv_done.notify_all();
    return AFD_OK;
  }

  void fail_all(afd_status s) {
    std::lock_guard<std::mutex> lk(mu);
    fatal = s;
    fatal_text = last_error_text();
    for (auto& kv : reqs) {
      if (kv.second->state != 2) {
        kv.second->state = 2;
        kv.second->status = s;
        kv.second->t_done = Clock::now();
        st.failed += 1;
      }
    }
    queue.clear();
    for (auto& sl : slots) {
      if (sl.used) arena.release(sl.block, sl.bytes);
      sl = Slot{};
    }
    n_active = 0;
    cv_done.notify_all();
  }

  void run() {
    DeviceScope scope(device);
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !queue.empty() || n_active > 0; });
        if (stop) return;
        afd_status s = admit();
        if (s != AFD_OK) {
          lk.unlock();
          fail_all(s);
          continue;
        }
        if (n_active == 0 && !queue.empty()) {
          // Nothing runs, yet the oldest request does not fit: memory is held
          // by free blocks of other sizes or by cached plans.  Return it all
          // and try once more; if it still does not fit, fail that request.
          (void)cudaStreamSynchronize(stream);
          for (auto& kv : plans) arena.uncharge(kv.second->bytes);
          plans.clear();
          arena.reset();
          s = admit();
          if (s == AFD_OK && n_active == 0 && !queue.empty()) {
            Request& r = *reqs[queue.front()];
            r.state = 2;
            r.status = AFD_ERR_BUDGET;
            r.t_done = Clock::now();
            queue.pop_front();
            st.failed += 1;
            cv_done.notify_all();
          }
          if (s != AFD_OK) {
            lk.unlock();
            fail_all(s);
          }
          continue;
        }
      }
      afd_status s = tick();
      if (s == AFD_OK) s = retire();
      if (s == AFD_OK) s = evict();
      if (s != AFD_OK) fail_all(s);
    }
  }
};

extern "C" {

afd_status afd_serve_create(afd_server** out, size_t mem_budget_bytes, const afd_plan_opts* opts) {
  clear_last_error();
  if (!out) return set_error(AFD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (mem_budget_bytes < (size_t(1) << 20))
    return set_error(AFD_ERR_INVALID, "mem_budget_bytes must be at least 1 MiB");
  afd_plan_opts o;
  int dev = 0;
  AFD_TRY(normalise_opts(opts, o, dev));
  if (o.offgrid_iters) return set_error(AFD_ERR_INVALID, "offgrid_iters: plans only");
  DeviceScope scope(dev);
  if (!scope.ok) return set_error(AFD_ERR_CUDA, "cannot make device %d current", dev);
  AFD_TRY(ensure_configured(dev));
  std::unique_ptr<afd_server> s(new (std::nothrow) afd_server(mem_budget_bytes));
  if (!s) return set_error(AFD_ERR_NOMEM, "host allocation failed");
  s->device = dev;
  s->opts = o;
  if (o.stream) {
    s->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    CUDA_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  s->slots.assign(kMaxSlots, Slot{});
  CUDA_TRY(cudaMalloc(&s->slots_dev, sizeof(SlotDev) * kMaxSlots));
  CUDA_TRY(cudaMalloc(&s->ctl_dev, sizeof(SlotCtl) * kMaxSlots));
  CUDA_TRY(cudaMalloc(&s->ids_dev, sizeof(int) * 2 * kMaxSlots));
  CUDA_TRY(cudaMalloc(&s->bar_dev, BAR_BYTES));
  CUDA_TRY(cudaMallocHost((void**)&s->slotdev_host, sizeof(SlotDev) * kMaxSlots));
  CUDA_TRY(cudaMallocHost((void**)&s->ctl_host, sizeof(SlotCtl) * kMaxSlots));
  CUDA_TRY(cudaMallocHost((void**)&s->ids_host, sizeof(int) * 2 * kMaxSlots));
  CUDA_TRY(cudaMemset(s->ctl_dev, 0, sizeof(SlotCtl) * kMaxSlots));
  const size_t fixed =
      sizeof(SlotDev) * kMaxSlots + sizeof(SlotCtl) * kMaxSlots + sizeof(int) * 2 * kMaxSlots + BAR_BYTES;
  if (!s->arena.charge(fixed)) return set_error(AFD_ERR_BUDGET, "budget below the fixed slot tables");
  s->fixed_bytes = fixed;
  afd_server* raw = s.get();
  s->worker = std::thread([raw] { raw->run(); });
  *out = s.release();
  return AFD_OK;
}

afd_status afd_serve_submit(afd_server* s, int N, const double* radii, int M, const double* G, int K_max,
                            double energy_tol, uint64_t* req_id) {
  clear_last_error();
  if (!s || !G || !req_id) return set_error(AFD_ERR_INVALID, "server, G or req_id is NULL");
  AFD_TRY(check_size(N, s->opts.precision));
  AFD_TRY(check_radii(radii, M));
  if (K_max < 1 || K_max > (1 << 16)) return set_error(AFD_ERR_INVALID, "K_max = %d out of range", K_max);
  if (!(energy_tol >= 0.0)) return set_error(AFD_ERR_INVALID, "energy_tol must be >= 0");
  if (s->opts.force_a1_zero && radii[0] != 0.0)
    return set_error(AFD_ERR_INVALID, "force_a1_zero needs radii[0] == 0");
  const int prec = s->opts.precision, cap = prec == AFD_FP32_GUARDED ? s->opts.guard_cap : 1;
  const size_t need = Arena::class_size(slot_layout(N, M, K_max, prec, cap).total);
  if (need + Tables::bytes_for(N, M, prec) + s->fixed_bytes > s->arena.budget())
    return set_error(AFD_ERR_BUDGET, "request needs %zu bytes, more than the budget", need);
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return set_error(AFD_ERR_NOMEM, "host allocation failed");
  r->N = N;
  r->K = K_max;
  r->tol = energy_tol;
  r->radii.assign(radii, radii + M);
  r->G.resize(2 * (size_t)N);
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, G) == cudaSuccess &&
      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
    DeviceScope scope(s->device);
    CUDA_TRY(cudaMemcpy(r->G.data(), G, 16 * (size_t)N, cudaMemcpyDeviceToHost));
  } else {
    cudaGetLastError();
    std::memcpy(r->G.data(), G, 16 * (size_t)N);
  }
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != AFD_OK) return set_error(s->fatal, "server failed earlier: %s", s->fatal_text.c_str());
  r->id = s->next_id++;
  *req_id = r->id;
  s->queue.push_back(r->id);
  s->reqs.emplace(r->id, std::move(r));
  s->st.submitted += 1;
  s->cv_work.notify_one();
  return AFD_OK;
}

static afd_status fill_result(Request& r, afd_result* out) {
  if (!out) return r.status;
  out->steps = r.steps;
  out->status = r.status;
  out->latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  if (out->K_cap < r.steps)
    return set_error(AFD_ERR_INVALID, "result arrays hold %d steps, the request made %d", out->K_cap, r.steps);
  if (out->delta) out->delta[0] = 1.0;
  for (int k = 0; k < r.steps; ++k) {
    const StepRec& q = r.recs[k];
    if (out->a) { out->a[2 * k] = q.a_re; out->a[2 * k + 1] = q.a_im; }
    if (out->coeff) { out->coeff[2 * k] = q.c_re; out->coeff[2 * k + 1] = q.c_im; }
    if (out->delta) out->delta[k + 1] = q.delta;
    if (out->idx) { out->idx[2 * k] = q.s; out->idx[2 * k + 1] = q.j; }
  }
  return r.status;
}

afd_status afd_serve_poll(afd_server* s, uint64_t req_id, afd_result* out) {
  if (!s) return set_error(AFD_ERR_INVALID, "server is NULL");
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return set_error(AFD_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    if (it->second->state != 2) return AFD_PENDING;
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  return fill_result(*r, out);
}

afd_status afd_serve_wait(afd_server* s, uint64_t req_id, double timeout_s, afd_result* out) {
  if (!s) return set_error(AFD_ERR_INVALID, "server is NULL");
  std::unique_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto pred = [&] {
      auto it = s->reqs.find(req_id);
      return it == s->reqs.end() || it->second->state == 2;
    };
    const auto limit = std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0);
    if (!s->cv_done.wait_for(lk, limit, pred)) return set_error(AFD_ERR_TIMEOUT, "request still running");
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return set_error(AFD_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  return fill_result(*r, out);
}

afd_status afd_serve_suspend(afd_server* s, uint64_t req_id, double timeout_s) {
  if (!s) return set_error(AFD_ERR_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return set_error(AFD_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
  Request& r = *it->second;
  if (r.state == 3) return AFD_OK;
  if (r.state == 2) return set_error(AFD_ERR_INVALID, "request %llu has finished", (unsigned long long)req_id);
  if (r.state == 0) {  // still queued: nothing on the device yet
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), req_id));
    r.state = 3;
    return AFD_OK;
  }
  r.suspend = true;
  s->cv_work.notify_one();
  auto pred = [&] {
    auto i2 = s->reqs.find(req_id);
    return i2 == s->reqs.end() || i2->second->state != 1;
  };
  const auto limit = std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0);
  if (!s->cv_done.wait_for(lk, limit, pred)) return set_error(AFD_ERR_TIMEOUT, "request still in its slot");
  auto i3 = s->reqs.find(req_id);
  if (i3 == s->reqs.end() || i3->second->state == 2)
    return set_error(AFD_ERR_INVALID, "request %llu finished before it could be suspended", (unsigned long long)req_id);
  return AFD_OK;
}

afd_status afd_serve_resume(afd_server* s, uint64_t req_id) {
  if (!s) return set_error(AFD_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return set_error(AFD_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
  if (it->second->state != 3) return set_error(AFD_ERR_INVALID, "request %llu is not suspended", (unsigned long long)req_id);
  it->second->state = 0;
  s->queue.push_back(req_id);
  s->cv_work.notify_one();
  return AFD_OK;
}

afd_status afd_serve_get_stats(afd_server* s, afd_serve_stats* out) {
  if (!s || !out) return set_error(AFD_ERR_INVALID, "server or out is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = (int)s->queue.size();
  out->active = s->n_active;
  out->bytes_reserved = s->arena.reserved();
  out->bytes_in_use = s->arena.in_use();
  return AFD_OK;
}

afd_status afd_serve_destroy(afd_server* s) {
  if (!s) return AFD_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  {
    DeviceScope scope(s->device);
    cudaStreamSynchronize(s->stream);
    s->plans.clear();
    delete s;
  }
  return AFD_OK;
}

}  // extern "C"
