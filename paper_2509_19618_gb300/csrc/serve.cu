// Request executor (include/hpmxp_serve.h): independent systems solved
// concurrently on one GPU.  Host code only; every step of a request is the
// library's own entry points (hpmxp_generate, hpmxp_factor, hpmxp_solve_ir)
// on the worker's stream.
#include "internal.h"
#include "../../include/hpmxp_serve.h"
#include "../../include/hpmxp_testing.h"

#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace hpmxp {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t kNone = ~(size_t)0;
constexpr int64_t kMaxRhs = 8;   // right-hand sides one solve refines together

// First-fit sub-allocator of [0, bytes): host bookkeeping of device memory.
// Free blocks are kept by offset and merged with their neighbours on release.
class Arena {
 public:
  explicit Arena(size_t bytes) : bytes_(bytes / kAlign * kAlign) {
    if (bytes_) free_[0] = bytes_;
  }
  size_t alloc(size_t n) {
    n = round_up(n, kAlign);
    if (n == 0) n = kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, left = it->second - n;
      free_.erase(it);
      if (left) free_[off + n] = left;
      return off;
    }
    return kNone;
  }
  void release(size_t off, size_t n) {
    n = round_up(n, kAlign);
    if (n == 0) n = kAlign;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {   // merge with the block after
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {                            // and with the block before
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }
  size_t capacity() const { return bytes_; }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto& kv : free_) s += kv.second;
    return s;
  }

 private:
  size_t bytes_;
  std::map<size_t, size_t> free_;
};

// Byte offsets of a request's buffers inside its arena block.
struct Layout {
  size_t lu = 0, fws = 0, sws = 0, a = 0, b = 0, x = 0, total = 0;
  size_t fws_bytes = 0, sws_bytes = 0;
  int64_t ld = 0;   // leading dimension of every n-row buffer the executor places
  int nb = 0;
};

int pick_nb(const hpmxp_request& r) { return r.nb ? r.nb : (r.n < 4096 ? 128 : 256); }

bool request_ok(const hpmxp_request& r) {
  if (r.n < 1 || r.n > (int64_t(1) << 17) || r.nrhs < 1 || r.nrhs > kMaxRhs) return false;
  if (!(r.prec >= HPMXP_BF16 && r.prec <= HPMXP_FP16_TRAIL32)) return false;
  const int nb = pick_nb(r);
  if (!(nb == 128 || nb == 256 || nb == 512)) return false;
  if ((r.A == nullptr) != (r.b == nullptr)) return false;
  if (r.A && (r.lda < r.n || r.ldb < r.n)) return false;
  if (!r.A && (r.diag_mode < HPMXP_DIAG_DOMINANT || r.diag_mode > HPMXP_DIAG_DEPARTURE)) return false;
  if (r.x && r.ldx < r.n) return false;
  const hpmxp_ir_params& p = r.params;
  if (p.restart < 1 || p.restart > 64 || p.max_iters < 0) return false;
  return true;
}

Layout layout(const hpmxp_request& r) {
  Layout L;
  L.nb = pick_nb(r);
  L.ld = round_up<int64_t>(r.n, 8);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += round_up(bytes, kAlign);
    return at;
  };
  L.lu = take(2 * (size_t)L.ld * (size_t)r.n);
  L.fws_bytes = factor_ws_bytes(r.n, r.prec, L.nb);
  L.fws = take(L.fws_bytes);
  // the solve workspace also serves generation (16 n bytes), which is done before the solve starts
  L.sws_bytes = std::max(solve_ws_bytes(r.n, r.nrhs, r.params.restart), round_up<size_t>(16 * (size_t)r.n, kAlign));
  L.sws = take(L.sws_bytes);
  if (!r.A) {
    L.a = take(8 * (size_t)L.ld * (size_t)r.n);
    L.b = take(8 * (size_t)L.ld * (size_t)r.nrhs);
  }
  if (!r.x) L.x = take(8 * (size_t)L.ld * (size_t)r.nrhs);
  L.total = off;
  return L;
}

struct Job {
  hpmxp_request r;
  Layout L;
  double t_submit;
};

// Batch mode: requests that can share the batched entry points (16-bit
// factors at depth 128 and the same refinement parameters).
bool batchable(const hpmxp_request& r) {
  return (r.prec == HPMXP_BF16 || r.prec == HPMXP_FP16) && (r.nb == 0 || r.nb == 128);
}
bool same_batch(const hpmxp_request& a, const hpmxp_request& b) {
  return a.prec == b.prec && memcmp(&a.params, &b.params, sizeof(hpmxp_ir_params)) == 0;
}

// One arena block for a batch: every request's LU, generated A and b, and x,
// then the batched factorization's and solve's workspaces.
struct BatchLayout {
  std::vector<size_t> lu, a, b, x;
  std::vector<int64_t> ld;
  size_t fws = 0, fws_bytes = 0, sws = 0, sws_bytes = 0, total = 0;
};

BatchLayout batch_layout(const std::vector<Job>& jobs, std::vector<hpmxp_problem>* probs_out) {
  BatchLayout B;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += round_up(std::max<size_t>(bytes, 1), kAlign);
    return at;
  };
  std::vector<hpmxp_problem> probs(jobs.size());
  for (size_t q = 0; q < jobs.size(); ++q) {
    const hpmxp_request& r = jobs[q].r;
    const int64_t ld = round_up<int64_t>(r.n, 8);
    B.ld.push_back(ld);
    B.lu.push_back(take(2 * (size_t)ld * (size_t)r.n));
    B.a.push_back(r.A ? kNone : take(8 * (size_t)ld * (size_t)r.n));
    B.b.push_back(r.A ? kNone : take(8 * (size_t)ld * (size_t)r.nrhs));
    B.x.push_back(r.x ? kNone : take(8 * (size_t)ld * (size_t)r.nrhs));
    probs[q] = hpmxp_problem{r.n, nullptr, ld, nullptr, ld, nullptr, ld, nullptr, ld, r.nrhs};
  }
  B.fws_bytes = factor_batched_ws_bytes(probs.data(), (int)probs.size());
  B.fws = take(B.fws_bytes);
  size_t gen = 0;
  for (const Job& j : jobs) gen = std::max<size_t>(gen, 16 * (size_t)j.r.n);
  // the solve workspace also serves generation (16 n bytes), done before the solve starts
  B.sws_bytes = std::max(solve_batched_ws_bytes(probs.data(), (int)probs.size(), jobs[0].r.params.restart),
                         round_up<size_t>(gen, kAlign));
  B.sws = take(B.sws_bytes);
  B.total = off;
  if (probs_out) *probs_out = probs;
  return B;
}

}  // namespace
}  // namespace hpmxp

using namespace hpmxp;

struct hpmxp_executor {
  int device = 0;
  int max_batch = 1;   // > 1: batch mode
  char* arena_base = nullptr;
  Arena arena{0};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::deque<hpmxp_completion> done;
  std::vector<std::thread> threads;
  int64_t outstanding = 0;
  bool stopping = false;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double clock() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  hpmxp_completion run(const Job& job, char* blk, cudaStream_t st) {
    const hpmxp_request& r = job.r;
    const Layout& L = job.L;
    hpmxp_completion c{};
    c.id = r.id;
    c.nrhs = (int)r.nrhs;
    c.t_submit = job.t_submit;
    c.t_start = clock();
    void* LU = blk + L.lu;
    void* fws = blk + L.fws;
    void* sws = blk + L.sws;
    const double* A = r.A;
    const double* b = r.b;
    int64_t lda = r.lda, ldb = r.ldb;
    double* x = r.x;
    int64_t ldx = r.ldx;
    hpmxp_status s = HPMXP_OK;
    if (!A) {
      double* Ag = (double*)(blk + L.a);
      double* bg = (double*)(blk + L.b);
      s = hpmxp_generate(r.n, r.seed, r.margin, r.diag_mode, Ag, L.ld, bg, L.ld, r.nrhs, sws, L.sws_bytes, st);
      A = Ag; b = bg; lda = L.ld; ldb = L.ld;
    }
    if (!x) {
      x = (double*)(blk + L.x);
      ldx = L.ld;
    }
    if (s == HPMXP_OK) s = hpmxp_factor(r.n, A, lda, r.prec, L.nb, LU, L.ld, fws, L.fws_bytes, st);
    if (s == HPMXP_OK)
      s = hpmxp_solve_ir(r.n, A, lda, LU, L.ld, r.prec, b, ldb, x, ldx, r.nrhs, &r.params, c.info, sws,
                         L.sws_bytes, st);
    else
      host_wait(st);   // nothing of this request may still run when its block is released
    c.status = (int32_t)s;
    c.t_done = clock();
    return c;
  }

  // A batch of requests through the batched entry points, in one arena block.
  std::vector<hpmxp_completion> run_batch(const std::vector<Job>& jobs, const BatchLayout& B, char* blk,
                                          cudaStream_t st) {
    const double t_start = clock();
    std::vector<hpmxp_problem> probs(jobs.size());
    hpmxp_status s = HPMXP_OK;
    for (size_t q = 0; q < jobs.size(); ++q) {
      const hpmxp_request& r = jobs[q].r;
      hpmxp_problem& p = probs[q];
      p.n = r.n; p.nrhs = r.nrhs;
      p.LU = blk + B.lu[q]; p.ldlu = B.ld[q];
      if (r.A) {
        p.A = r.A; p.lda = r.lda; p.b = r.b; p.ldb = r.ldb;
      } else {
        double* Ag = (double*)(blk + B.a[q]);
        double* bg = (double*)(blk + B.b[q]);
        if (s == HPMXP_OK)
          s = hpmxp_generate(r.n, r.seed, r.margin, r.diag_mode, Ag, B.ld[q], bg, B.ld[q], r.nrhs, blk + B.sws,
                             B.sws_bytes, st);
        p.A = Ag; p.lda = B.ld[q]; p.b = bg; p.ldb = B.ld[q];
      }
      if (r.x) { p.x = r.x; p.ldx = r.ldx; } else { p.x = (double*)(blk + B.x[q]); p.ldx = B.ld[q]; }
    }
    std::vector<hpmxp_status> fst(jobs.size(), HPMXP_OK);
    if (s == HPMXP_OK)
      hpmxp_factor_batched(probs.data(), (int)probs.size(), jobs[0].r.prec, fst.data(), blk + B.fws, B.fws_bytes,
                           st);
    // systems whose factorization broke down are reported and left out of the solve
    std::vector<hpmxp_problem> good;
    std::vector<size_t> idx;
    for (size_t q = 0; q < jobs.size(); ++q)
      if (s == HPMXP_OK && fst[q] == HPMXP_OK) { good.push_back(probs[q]); idx.push_back(q); }
    std::vector<hpmxp_ir_info> info;
    for (const hpmxp_problem& p : good) info.resize(info.size() + (size_t)p.nrhs);
    if (!good.empty())
      hpmxp_solve_ir_batched(good.data(), (int)good.size(), jobs[0].r.prec, &jobs[0].r.params, info.data(),
                             blk + B.sws, B.sws_bytes, st);
    host_wait(st);   // nothing of the batch may still run when its block is released
    const double t_done = clock();
    std::vector<hpmxp_completion> out(jobs.size());
    size_t off = 0, gi = 0;
    for (size_t q = 0; q < jobs.size(); ++q) {
      hpmxp_completion& c = out[q];
      c = hpmxp_completion{};
      c.id = jobs[q].r.id;
      c.nrhs = (int)jobs[q].r.nrhs;
      c.t_submit = jobs[q].t_submit;
      c.t_start = t_start;
      c.t_done = t_done;
      if (s != HPMXP_OK) { c.status = s; continue; }
      if (fst[q] != HPMXP_OK) { c.status = fst[q]; continue; }
      int worst = HPMXP_OK;
      for (int r = 0; r < c.nrhs; ++r) {
        c.info[r] = info[off + r];
        if (info[off + r].status != HPMXP_OK && worst == HPMXP_OK) worst = info[off + r].status;
      }
      c.status = worst;
      off += (size_t)c.nrhs;
      ++gi;
    }
    return out;
  }

  void worker() {
    cudaStream_t st = nullptr;
    const bool ok = cudaSetDevice(device) == cudaSuccess &&
                    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    if (max_batch > 1) {
      batch_worker(st, ok);
      if (st) cudaStreamDestroy(st);
      return;
    }
    for (;;) {
      Job job;
      size_t off = kNone;
      {
        std::unique_lock<std::mutex> lk(mu);
        // strict arrival order: the head is admitted once its block fits
        cv_work.wait(lk, [&] {
          if (queue.empty()) return stopping;
          off = arena.alloc(queue.front().L.total);
          return off != kNone;
        });
        if (queue.empty()) break;
        job = queue.front();
        queue.pop_front();
        if (!queue.empty()) cv_work.notify_one();   // the next head may fit too
      }
      hpmxp_completion c;
      if (ok) {
        c = run(job, arena_base + off, st);
      } else {
        c = hpmxp_completion{};
        c.id = job.r.id;
        c.nrhs = (int)job.r.nrhs;
        c.t_submit = job.t_submit;
        c.t_start = c.t_done = clock();
        c.status = HPMXP_ECUDA;
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        arena.release(off, job.L.total);
        done.push_back(c);
      }
      cv_work.notify_all();
      cv_done.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  }

  // Batch mode: the head of the queue and the requests after it (arrival
  // order, up to max_batch, batchable and of the same kind) whose batch block
  // fits the arena; a request that cannot be batched runs alone.
  void batch_worker(cudaStream_t st, bool ok) {
    for (;;) {
      std::vector<Job> jobs;
      BatchLayout B;
      size_t off = kNone;
      bool single = false;
      Layout L1;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (queue.empty()) return stopping;
          const Job& head = queue.front();
          if (!batchable(head.r)) {
            off = arena.alloc(head.L.total);
            single = true;
            return off != kNone;
          }
          single = false;
          std::vector<Job> cand;
          for (size_t i = 0; i < queue.size() && (int)cand.size() < max_batch; ++i) {
            if (!batchable(queue[i].r) || !same_batch(queue[i].r, head.r)) break;
            cand.push_back(queue[i]);
          }
          while (!cand.empty()) {
            BatchLayout trial = batch_layout(cand, nullptr);
            off = arena.alloc(trial.total);
            if (off != kNone) { jobs = cand; B = trial; return true; }
            cand.pop_back();
          }
          return false;
        });
        if (queue.empty()) break;
        if (single) {
          jobs.push_back(queue.front());
          L1 = queue.front().L;
          queue.pop_front();
        } else {
          for (size_t i = 0; i < jobs.size(); ++i) queue.pop_front();
        }
        if (!queue.empty()) cv_work.notify_one();
      }
      std::vector<hpmxp_completion> cs;
      if (!ok) {
        for (const Job& j : jobs) {
          hpmxp_completion c{};
          c.id = j.r.id; c.nrhs = (int)j.r.nrhs; c.t_submit = j.t_submit; c.t_start = c.t_done = clock();
          c.status = HPMXP_ECUDA;
          cs.push_back(c);
        }
      } else if (single) {
        cs.push_back(run(jobs[0], arena_base + off, st));
      } else {
        cs = run_batch(jobs, B, arena_base + off, st);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        arena.release(off, single ? L1.total : B.total);
        for (auto& c : cs) done.push_back(c);
      }
      cv_work.notify_all();
      cv_done.notify_all();
    }
  }
};

extern "C" {

size_t hpmxp_request_footprint(const hpmxp_request* r) {
  if (!r || !request_ok(*r)) return 0;
  return layout(*r).total;
}

namespace {
hpmxp_status create_executor(int device, int workers, int max_batch, void* arena, size_t arena_bytes,
                             hpmxp_executor** out) {
  if (!out || workers < 1 || workers > 64 || max_batch < 1 || max_batch > 256 || !arena ||
      ((uintptr_t)arena % kAlign) != 0 || arena_bytes < kAlign)
    return HPMXP_EINVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return HPMXP_EINVAL;
  hpmxp_executor* ex = new hpmxp_executor();
  ex->device = device;
  ex->max_batch = max_batch;
  ex->arena_base = (char*)arena;
  ex->arena = Arena(arena_bytes);
  for (int i = 0; i < workers; ++i) ex->threads.emplace_back([ex] { ex->worker(); });
  *out = ex;
  return HPMXP_OK;
}
}  // namespace

hpmxp_status hpmxp_executor_create(int device, int workers, void* arena, size_t arena_bytes,
                                   hpmxp_executor** out) {
  return create_executor(device, workers, 1, arena, arena_bytes, out);
}

hpmxp_status hpmxp_executor_create_batched(int device, int workers, int max_batch, void* arena, size_t arena_bytes,
                                           hpmxp_executor** out) {
  return create_executor(device, workers, max_batch, arena, arena_bytes, out);
}

hpmxp_status hpmxp_executor_submit(hpmxp_executor* ex, const hpmxp_request* r) {
  if (!ex || !r || !request_ok(*r)) return HPMXP_EINVAL;
  Job job{*r, layout(*r), 0.0};
  if (job.L.total > ex->arena.capacity()) return HPMXP_ENOMEM;
  if (ex->max_batch > 1 && batchable(*r) && batch_layout({job}, nullptr).total > ex->arena.capacity())
    return HPMXP_ENOMEM;
  {
    std::lock_guard<std::mutex> lk(ex->mu);
    if (ex->stopping) return HPMXP_EINVAL;
    job.t_submit = ex->clock();
    ex->queue.push_back(job);
    ++ex->outstanding;
  }
  ex->cv_work.notify_one();
  return HPMXP_OK;
}

int hpmxp_executor_poll(hpmxp_executor* ex, hpmxp_completion* out, int max, int timeout_ms) {
  if (!ex || !out || max < 1) return 0;
  std::unique_lock<std::mutex> lk(ex->mu);
  if (ex->done.empty() && timeout_ms > 0)
    ex->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !ex->done.empty(); });
  int k = 0;
  while (k < max && !ex->done.empty()) {
    out[k++] = ex->done.front();
    ex->done.pop_front();
    --ex->outstanding;
  }
  return k;
}

int64_t hpmxp_executor_outstanding(hpmxp_executor* ex) {
  if (!ex) return 0;
  std::lock_guard<std::mutex> lk(ex->mu);
  return ex->outstanding;
}

double hpmxp_executor_clock(hpmxp_executor* ex) { return ex ? ex->clock() : 0.0; }

hpmxp_status hpmxp_executor_destroy(hpmxp_executor* ex) {
  if (!ex) return HPMXP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(ex->mu);
    ex->stopping = true;
  }
  ex->cv_work.notify_all();
  for (auto& t : ex->threads) t.join();
  delete ex;
  return HPMXP_OK;
}

// Host-only check of the arena: ops[i] > 0 allocates that many bytes
// (result[i] = offset or -1), ops[i] = -(k + 1) releases the block of op k
// (result[i] = bytes free afterwards).
int hpmxp_test_arena(size_t arena_bytes, const int64_t* ops, int nops, int64_t* result) {
  if (!ops || !result || nops < 0) return HPMXP_EINVAL;
  Arena a(arena_bytes);
  for (int i = 0; i < nops; ++i) {
    if (ops[i] > 0) {
      const size_t off = a.alloc((size_t)ops[i]);
      result[i] = off == kNone ? -1 : (int64_t)off;
    } else {
      const int64_t k = -ops[i] - 1;
      if (k < 0 || k >= i || ops[k] <= 0 || result[k] < 0) return HPMXP_EINVAL;
      a.release((size_t)result[k], (size_t)ops[k]);
      result[i] = (int64_t)a.free_bytes();
    }
  }
  return HPMXP_OK;
}

}  // extern "C"
