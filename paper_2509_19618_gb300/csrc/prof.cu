// Measurement support (not part of the paper's method): a count of this
// library's kernel launches, and optional CUDA-event timing of selected
// kernels on the stream that launches them, so a benchmark can attribute
// time and work to the dominant kernel without a profiler.
#include "internal.h"

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

namespace hpmxp {

namespace {
std::atomic<int> g_tile{0}, g_reserve{0}, g_budget{0};
std::atomic<long long> g_overlap{0};
thread_local int t_budget = 0;
}  // namespace

SmBudgetScope::SmBudgetScope(int sms) : prev(t_budget) { t_budget = sms; }
SmBudgetScope::~SmBudgetScope() { t_budget = prev; }

int sm_budget() {
  static const int env_budget = [] {
    const char* e = getenv("HPMXP_SM_BUDGET");
    return e ? atoi(e) : 0;
  }();
  if (t_budget > 0) return t_budget;
  if (env_budget > 0) return env_budget;
  return g_budget.load();
}

// The tile override is read once (the value is consulted per GEMM launch);
// the two schedule overrides are read per factorization.
hpmxp_tuning tuning() {
  static const int env_tile = [] {
    const char* e = getenv("HPMXP_GEMM_TILE");
    return e ? atoi(e) : 0;
  }();
  hpmxp_tuning t{g_tile.load(), g_reserve.load(), g_overlap.load(), g_budget.load(), 0};
  if (env_tile) t.gemm_tile = env_tile;
  if (const char* e = getenv("HPMXP_RESERVE_SMS")) t.reserve_sms = atoi(e);
  if (const char* e = getenv("HPMXP_OVERLAP_MIN")) t.overlap_min = atoll(e);
  return t;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("HPMXP_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

namespace {

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_enabled{0};

struct Span {
  cudaEvent_t a, b;
  int kind;
  double work, bytes;
  int slot;                           // device span slot (-1: none)
};

std::mutex g_mu;
std::vector<Span> g_open;             // recorded, not yet resolved
cudaEvent_t g_origin = nullptr;       // first span start since the last reset
struct Interval {
  int kind;
  double t0, t1;                      // ms after g_origin
};
std::vector<Interval> g_timeline;     // resolved spans, in recording order
constexpr size_t kMaxTimeline = size_t(1) << 20;
double g_ms[kProfKinds], g_work[kProfKinds], g_bytes[kProfKinds];
long long g_count[kProfKinds];
std::vector<cudaEvent_t> g_pool;
// Device spans of the kernels that record their own execution (first CTA start
// to last CTA end on the global timer): a ring of slot pairs on one device,
// all-ones when unused; token -> slot for the launch between prof_begin and
// prof_end.
constexpr int kSpanSlots = 1 << 16;
unsigned long long* g_span_dev = nullptr;
int g_span_device = -1;
int g_span_next = 0;
std::vector<std::pair<void*, int>> g_span_of;
double g_dev_ms[kProfKinds];
long long g_dev_count[kProfKinds];

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void resolve_locked() {
  std::vector<unsigned long long> spans;
  for (const Span& s : g_open)
    if (s.slot >= 0 && spans.empty()) {
      spans.resize(2 * (size_t)g_span_next);
      if (cudaMemcpy(spans.data(), g_span_dev, sizeof(unsigned long long) * spans.size(), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
        spans.clear();
    }
  for (Span& s : g_open) {
    float ms = 0.0f;
    if (cudaEventSynchronize(s.b) == cudaSuccess && cudaEventElapsedTime(&ms, s.a, s.b) == cudaSuccess) {
      g_ms[s.kind] += ms;
      g_work[s.kind] += s.work;
      g_bytes[s.kind] += s.bytes;
      g_count[s.kind] += 1;
      float t0 = 0.0f;
      if (g_origin && g_timeline.size() < kMaxTimeline && cudaEventElapsedTime(&t0, g_origin, s.a) == cudaSuccess)
        g_timeline.push_back(Interval{s.kind, (double)t0, (double)t0 + ms});
      if (s.slot >= 0 && 2 * (size_t)s.slot + 1 < spans.size()) {
        const unsigned long long t_start = spans[2 * (size_t)s.slot], t_end = ~spans[2 * (size_t)s.slot + 1];
        if (t_start != ~0ull && t_end != 0ull && t_end >= t_start) {
          g_dev_ms[s.kind] += (double)(t_end - t_start) * 1e-6;
          g_dev_count[s.kind] += 1;
        }
      }
    }
    if (s.a != g_origin) g_pool.push_back(s.a);
    g_pool.push_back(s.b);
  }
  g_open.clear();
}

}  // namespace

// Host waits of the library.  By default the calling thread spins in
// cudaStreamSynchronize (lowest latency); HPMXP_BLOCKING_WAIT=1 makes it
// sleep on a blocking-sync event instead, which frees host cores when many
// threads each drive their own stream but adds a wake-up delay to every wait.
cudaError_t host_wait(cudaStream_t st) {
  static const bool blocking = [] {
    const char* e = getenv("HPMXP_BLOCKING_WAIT");
    return e && e[0] == '1';
  }();
  if (!blocking) return cudaStreamSynchronize(st);
  struct Events {
    cudaEvent_t ev[64] = {};
    ~Events() {
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
  };
  thread_local Events tl;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaStreamSynchronize(st);
  cudaEvent_t& ev = tl.ev[dev];
  if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming)) != cudaSuccess) {
    ev = nullptr;
    return e;
  }
  if ((e = cudaEventRecord(ev, st)) != cudaSuccess) return e;
  return cudaEventSynchronize(ev);
}

// Device -> host read of `bytes` through a per-thread pinned staging buffer
// (a copy into pageable memory would wait inside the driver, spinning), then
// host_wait.  Returns once `dst` holds the data.
cudaError_t read_to_host(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  struct Staging {
    void* p = nullptr;
    size_t cap = 0;
    ~Staging() {
      if (p) cudaFreeHost(p);
    }
  };
  thread_local Staging tl;
  if (tl.cap < bytes) {
    if (tl.p) cudaFreeHost(tl.p);
    tl.p = nullptr;
    tl.cap = 0;
    const size_t cap = std::max<size_t>(bytes, 4096);
    cudaError_t e = cudaMallocHost(&tl.p, cap);
    if (e != cudaSuccess) {
      tl.p = nullptr;
      return e;
    }
    tl.cap = cap;
  }
  cudaError_t e = cudaMemcpyAsync(tl.p, src, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = host_wait(st);
  if (e == cudaSuccess) memcpy(dst, tl.p, bytes);
  return e;
}

void count_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

bool prof_on() { return g_enabled.load(std::memory_order_relaxed) != 0; }

void* prof_begin(cudaStream_t st) {
  if (!prof_on()) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t a = take_event();
  cudaEventRecord(a, st);
  if (!g_origin) g_origin = a;     // kept out of the pool until the next reset
  return (void*)a;
}

unsigned long long* prof_device_span(void* token) {
  if (!token) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (!g_span_dev) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(unsigned long long) * 2 * kSpanSlots) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0xFF, sizeof(unsigned long long) * 2 * kSpanSlots) != cudaSuccess) {
      cudaFree(p);
      return nullptr;
    }
    g_span_dev = (unsigned long long*)p;
    g_span_device = dev;
    g_span_next = 0;
  }
  if (dev != g_span_device || g_span_next >= kSpanSlots) return nullptr;
  const int slot = g_span_next++;
  g_span_of.emplace_back(token, slot);
  return g_span_dev + 2 * (size_t)slot;
}

void prof_end(void* token, int kind, double work, cudaStream_t st, double bytes) {
  if (!token) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st);
  int slot = -1;
  for (size_t i = g_span_of.size(); i-- > 0;)
    if (g_span_of[i].first == token) {
      slot = g_span_of[i].second;
      g_span_of.erase(g_span_of.begin() + (long)i);
      break;
    }
  g_open.push_back(Span{(cudaEvent_t)token, b, kind, work, bytes, slot});
  if (g_open.size() > 4096) resolve_locked();
}

}  // namespace hpmxp

using namespace hpmxp;

extern "C" {

unsigned long long hpmxp_launch_count(void) { return g_launches.load(); }

hpmxp_status hpmxp_set_tuning(const hpmxp_tuning* t) {
  if (!t || !(t->gemm_tile == 0 || t->gemm_tile == 128 || t->gemm_tile == 256) || t->reserve_sms < 0 ||
      t->reserve_sms > 1024 || t->overlap_min < 0 || t->sm_budget < 0 || t->sm_budget > 1024 || t->reserved != 0)
    return HPMXP_EINVAL;
  g_tile.store(t->gemm_tile);
  g_reserve.store(t->reserve_sms);
  g_overlap.store(t->overlap_min);
  g_budget.store(t->sm_budget);
  return HPMXP_OK;
}

void hpmxp_get_tuning(hpmxp_tuning* t) {
  if (t) *t = hpmxp_tuning{g_tile.load(), g_reserve.load(), g_overlap.load(), g_budget.load(), 0};
}

void hpmxp_prof_enable(int on) { g_enabled.store(on ? 1 : 0); }

void hpmxp_prof_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  for (int k = 0; k < kProfKinds; ++k) {
    g_ms[k] = 0.0; g_work[k] = 0.0; g_bytes[k] = 0.0; g_count[k] = 0;
    g_dev_ms[k] = 0.0; g_dev_count[k] = 0;
  }
  // every recorded kernel has completed (resolve_locked waited for its end event)
  if (g_span_dev && g_span_next > 0) {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev == g_span_device)
      cudaMemset(g_span_dev, 0xFF, sizeof(unsigned long long) * 2 * (size_t)g_span_next);
    g_span_next = 0;
  }
  g_span_of.clear();
  if (g_origin) g_pool.push_back(g_origin);
  g_origin = nullptr;
  g_timeline.clear();
}

int hpmxp_prof_read_device(int kind, double* ms, long long* count) {
  if (kind < 0 || kind >= kProfKinds) return HPMXP_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  if (ms) *ms = g_dev_ms[kind];
  if (count) *count = g_dev_count[kind];
  return HPMXP_OK;
}

int hpmxp_prof_timeline(double* out, int max_spans) {
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  const int k = (int)std::min<size_t>(g_timeline.size(), max_spans > 0 ? (size_t)max_spans : 0);
  if (out) {
    for (int i = 0; i < k; ++i) {
      out[3 * i] = g_timeline[i].kind;
      out[3 * i + 1] = g_timeline[i].t0;
      out[3 * i + 2] = g_timeline[i].t1;
    }
  }
  return (int)g_timeline.size();
}

int hpmxp_prof_read_bytes(int kind, double* total_bytes) {
  if (kind < 0 || kind >= kProfKinds || !total_bytes) return HPMXP_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  *total_bytes = g_bytes[kind];
  return HPMXP_OK;
}

int hpmxp_prof_read(int kind, double* total_ms, double* total_work, long long* launches) {
  if (kind < 0 || kind >= kProfKinds || !total_ms || !total_work || !launches) return HPMXP_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  *total_ms = g_ms[kind];
  *total_work = g_work[kind];
  *launches = g_count[kind];
  return HPMXP_OK;
}

}  // extern "C"
