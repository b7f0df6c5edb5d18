// Native SPMD harness (gvm_spmd_run): one thread per rank runs the paper's
// per-process loop -- submit the task, wait at the request barrier, collect
// the result (Section 6) -- through the public API only, so that measured
// step times contain the manager's work and not an interpreter's.
#include <cuda_runtime.h>

#include <sys/prctl.h>

#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "gvm.h"

namespace {

// Reusable barrier for a fixed number of threads (generation counting; waits
// yield so that more threads than cores still make progress).
class SpinBarrier {
 public:
  explicit SpinBarrier(int n) : n_(n) {}
  void wait() {
    const uint32_t gen = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
      count_.store(0, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_acq_rel);
      return;
    }
    uint32_t spins = 0;
    const auto t0 = std::chrono::steady_clock::now();
    while (gen_.load(std::memory_order_acquire) == gen) {
      if (++spins <= 64) continue;
      // After 5 ms (longer than a step's launch), sleep between checks:
      // waiting threads free the cores for the threads the barrier waits for.
      if ((spins & 63) == 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(5)) {
        thread_local bool slack_set = false;  // 1 us timer slack for this thread's short sleeps
        if (!slack_set) {
          prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
          slack_set = true;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(10));
      } else
        std::this_thread::yield();
    }
  }

 private:
  const int n_;
  std::atomic<int> count_{0};
  std::atomic<uint32_t> gen_{0};
};

// Submits the whole batch, syncing the rank's oldest outstanding task when
// the ring or the staging space is full. Returns the last sequence number
// through *last.
int submit_batch(gvm_rank* r, const gvm_task* tasks, uint32_t count, uint64_t* last) {
  uint32_t done = 0;
  uint64_t first_of_step = 0;
  bool have_first = false;
  while (done < count) {
    uint64_t first = 0;
    const int rc = gvm_submit_many(r, tasks + done, count - done, &first);
    if (rc < 0) return rc;
    if (rc > 0) {
      if (!have_first) {
        first_of_step = first;
        have_first = true;
      }
      done += (uint32_t)rc;
      *last = first + (uint64_t)rc - 1;
      continue;
    }
    // Nothing admitted: the ring is full of this step's earlier tasks.
    if (!have_first) return GVM_EAGAIN;
    const int s = gvm_sync(r, first_of_step);
    if (s != GVM_OK) return s;
    ++first_of_step;
  }
  return GVM_OK;
}

}  // namespace

extern "C" int gvm_spmd_run(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* tasks,
                            const uint32_t* counts, int32_t nranks, int32_t steps, float* step_ms_device,
                            float* launch_ms_device, double* step_ms_host, double* const* latency_ns) {
  if (!ctx || !ranks || !tasks || !counts || nranks <= 0 || steps < 0) return GVM_EINVAL;
  for (int r = 0; r < nranks; ++r)
    if (!ranks[r] || (counts[r] && !tasks[r])) return GVM_EINVAL;
  cudaStream_t sched = static_cast<cudaStream_t>(gvm_stream(ctx, -1));
  int dev = 0;
  if (!sched || cudaGetDevice(&dev) != cudaSuccess) return GVM_EINVAL;
  // Events per step: step start, step end, before and after the flush.
  std::vector<cudaEvent_t> ev;
  if (step_ms_device || launch_ms_device) {
    ev.resize(4 * (size_t)steps);
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        for (auto& x : ev)
          if (x) cudaEventDestroy(x);
        return GVM_EDEVICE;
      }
  }
  SpinBarrier bar(nranks);
  std::atomic<int> err{GVM_OK};
  std::vector<std::chrono::steady_clock::time_point> t0(steps), t1(steps);
  auto body = [&](int r) {
    cudaSetDevice(dev);
    double* lat = latency_ns ? latency_ns[r] : nullptr;
    for (int i = 0; i < steps; ++i) {
      if (r == 0) {
        t0[i] = std::chrono::steady_clock::now();
        if (!ev.empty() && cudaEventRecord(ev[4 * i], sched) != cudaSuccess) err.store(GVM_EDEVICE);
      }
      bar.wait();
      uint64_t last = 0;
      const auto t_submit = std::chrono::steady_clock::now();
      int rc = err.load() == GVM_OK && counts[r] ? submit_batch(ranks[r], tasks[r], counts[r], &last) : GVM_OK;
      if (rc != GVM_OK) {
        int ok = GVM_OK;
        err.compare_exchange_strong(ok, rc);
      }
      bar.wait();
      if (r == 0 && err.load() == GVM_OK) {
        if (!ev.empty()) cudaEventRecord(ev[4 * i + 2], sched);
        rc = gvm_flush(ctx);
        if (!ev.empty()) cudaEventRecord(ev[4 * i + 3], sched);
        if (rc != GVM_OK) {
          int ok = GVM_OK;
          err.compare_exchange_strong(ok, rc);
        }
      }
      bar.wait();
      if (err.load() == GVM_OK && counts[r] && lat) {
        // Collect the batch task by task, in submission order, recording
        // when each completion becomes visible to the rank.
        const uint64_t first = last + 1 - counts[r];
        for (uint32_t j = 0; j < counts[r] && err.load() == GVM_OK; ++j) {
          rc = gvm_sync(ranks[r], first + j);
          if (rc != GVM_OK) {
            int ok = GVM_OK;
            err.compare_exchange_strong(ok, rc);
            break;
          }
          lat[(size_t)i * counts[r] + j] =
              (double)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t_submit)
                  .count();
        }
      } else if (err.load() == GVM_OK && counts[r]) {
        rc = gvm_sync(ranks[r], last);
        if (rc != GVM_OK) {
          int ok = GVM_OK;
          err.compare_exchange_strong(ok, rc);
        }
      }
      bar.wait();
      if (r == 0) {
        if (!ev.empty() && cudaEventRecord(ev[4 * i + 1], sched) != cudaSuccess) err.store(GVM_EDEVICE);
        t1[i] = std::chrono::steady_clock::now();
      }
    }
  };
  std::vector<std::thread> th;
  th.reserve(nranks - 1);
  for (int r = 1; r < nranks; ++r) th.emplace_back(body, r);
  body(0);
  for (auto& t : th) t.join();
  int rc = err.load();
  if (!ev.empty()) {
    if (rc == GVM_OK && steps > 0 && cudaEventSynchronize(ev[4 * (steps - 1) + 1]) != cudaSuccess)
      rc = GVM_EDEVICE;
    for (int i = 0; rc == GVM_OK && i < steps; ++i) {
      if (step_ms_device && cudaEventElapsedTime(&step_ms_device[i], ev[4 * i], ev[4 * i + 1]) != cudaSuccess)
        rc = GVM_EDEVICE;
      if (launch_ms_device &&
          cudaEventElapsedTime(&launch_ms_device[i], ev[4 * i + 2], ev[4 * i + 3]) != cudaSuccess)
        rc = GVM_EDEVICE;
    }
    for (auto& e : ev) cudaEventDestroy(e);
  }
  if (step_ms_host)
    for (int i = 0; i < steps; ++i)
      step_ms_host[i] = std::chrono::duration<double, std::milli>(t1[i] - t0[i]).count();
  return rc;
}

extern "C" int gvm_spmd_run_pipelined(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* const* phases,
                                      int32_t nphases, const uint32_t* counts, int32_t nranks, int32_t steps,
                                      double* total_ms_host, double* done_ms_host) {
  if (!ctx || !ranks || !phases || nphases < 1 || !counts || nranks <= 0 || steps < 0 || !total_ms_host)
    return GVM_EINVAL;
  for (int p = 0; p < nphases; ++p)
    if (!phases[p]) return GVM_EINVAL;
  for (int r = 0; r < nranks; ++r) {
    if (!ranks[r]) return GVM_EINVAL;
    for (int p = 0; p < nphases; ++p)
      if (counts[r] && !phases[p][r]) return GVM_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GVM_EINVAL;
  SpinBarrier bar(nranks);
  std::atomic<int> err{GVM_OK};
  auto fail = [&](int rc) {
    int ok = GVM_OK;
    err.compare_exchange_strong(ok, rc);
  };
  const int lag = nphases - 1;  // steps submitted ahead of the one collected
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<std::chrono::steady_clock::time_point> t_done(steps);
  auto body = [&](int r) {
    cudaSetDevice(dev);
    std::vector<uint64_t> last(steps, 0);
    for (int i = 0; i < steps + lag; ++i) {
      // Step i: submit (every rank), meet, flush (thread 0), meet.
      if (i < steps) {
        const gvm_task* t = phases[i % nphases][r];
        if (err.load() == GVM_OK && counts[r]) {
          const int rc = submit_batch(ranks[r], t, counts[r], &last[i]);
          if (rc != GVM_OK) fail(rc);
        }
        bar.wait();
        if (r == 0 && err.load() == GVM_OK) {
          const int rc = gvm_flush(ctx);
          if (rc != GVM_OK) fail(rc);
        }
        bar.wait();
      }
      // Then the results of step i - lag.
      const int j = i - lag;
      if (j >= 0) {
        if (err.load() == GVM_OK && counts[r]) {
          const int rc = gvm_sync(ranks[r], last[j]);
          if (rc != GVM_OK) fail(rc);
        }
        bar.wait();
        if (r == 0) t_done[j] = std::chrono::steady_clock::now();
      }
    }
  };
  std::vector<std::thread> th;
  th.reserve(nranks - 1);
  for (int r = 1; r < nranks; ++r) th.emplace_back(body, r);
  body(0);
  for (auto& t : th) t.join();
  const auto t1 = std::chrono::steady_clock::now();
  *total_ms_host = std::chrono::duration<double, std::milli>(t1 - t0).count();
  if (done_ms_host)
    for (int i = 0; i < steps; ++i) done_ms_host[i] = std::chrono::duration<double, std::milli>(t_done[i] - t0).count();
  return err.load();
}

extern "C" int gvm_spmd_run_overlapped(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* tasks_even,
                                       const gvm_task* const* tasks_odd, const uint32_t* counts, int32_t nranks,
                                       int32_t steps, double* total_ms_host, double* done_ms_host) {
  if (!tasks_even) return GVM_EINVAL;
  const gvm_task* const* phases[2] = {tasks_even, tasks_odd ? tasks_odd : tasks_even};
  return gvm_spmd_run_pipelined(ctx, ranks, phases, 2, counts, nranks, steps, total_ms_host, done_ms_host);
}

extern "C" int gvm_open_loop_run(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* tasks,
                                 const uint64_t* const* arrival_ns, const uint32_t* counts, int32_t nranks,
                                 uint32_t max_inflight, double* const* latency_ns, double* span_ns) {
  if (!ctx || !ranks || !tasks || !arrival_ns || !counts || nranks <= 0 || !span_ns) return GVM_EINVAL;
  for (int r = 0; r < nranks; ++r) {
    if (!ranks[r] || (counts[r] && (!tasks[r] || !arrival_ns[r]))) return GVM_EINVAL;
    for (uint32_t i = 1; i < counts[r]; ++i)
      if (arrival_ns[r][i] < arrival_ns[r][i - 1]) return GVM_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GVM_EINVAL;
  using clk = std::chrono::steady_clock;
  std::atomic<int> err{GVM_OK};
  auto fail = [&](int rc) {
    int ok = GVM_OK;
    err.compare_exchange_strong(ok, rc);
  };
  const clk::time_point t0 = clk::now() + std::chrono::milliseconds(2);
  std::vector<clk::time_point> last(nranks, t0);
  auto ns_since = [&](clk::time_point t) { return (double)std::chrono::duration_cast<std::chrono::nanoseconds>(t - t0).count(); };
  auto body = [&](int r) {
    cudaSetDevice(dev);
    gvm_rank* rk = ranks[r];
    const uint32_t n = counts[r];
    std::vector<uint64_t> seq(n, 0);
    uint32_t next = 0, done = 0;  // tasks submitted, tasks seen complete
    auto seen = [&](uint32_t i) {
      const clk::time_point t = clk::now();
      if (latency_ns && latency_ns[r]) latency_ns[r][i] = ns_since(t) - (double)arrival_ns[r][i];
      last[r] = t;
    };
    auto reap_ready = [&]() {
      while (done < next) {
        const int p = gvm_poll(rk, seq[done]);
        if (p < 0) {
          fail(p);
          return;
        }
        if (p == 0) return;
        seen(done++);
      }
    };
    auto reap_one = [&]() {  // blocking: the oldest outstanding task
      const int s = gvm_sync(rk, seq[done]);
      if (s != GVM_OK) {
        fail(s);
        return;
      }
      seen(done++);
    };
    while (next < n && err.load() == GVM_OK) {
      const clk::time_point due = t0 + std::chrono::nanoseconds(arrival_ns[r][next]);
      // Until the arrival: collect completions, then wait (sleep when far).
      for (;;) {
        reap_ready();
        const clk::time_point now = clk::now();
        if (now >= due || err.load() != GVM_OK) break;
        if (due - now > std::chrono::microseconds(200))
          std::this_thread::sleep_for(std::chrono::microseconds(50));
        else
          std::this_thread::yield();
      }
      if (max_inflight && next - done >= max_inflight) reap_one();
      for (;;) {
        const int rc = gvm_submit(rk, &tasks[r][next], &seq[next]);
        if (rc == GVM_OK) break;
        if (rc != GVM_EAGAIN || done == next) {  // nothing of this rank left to wait for
          fail(rc);
          break;
        }
        reap_one();
        if (err.load() != GVM_OK) break;
      }
      if (err.load() != GVM_OK) break;
      ++next;
    }
    while (done < next && err.load() == GVM_OK) reap_one();
  };
  std::vector<std::thread> th;
  th.reserve(nranks - 1);
  for (int r = 1; r < nranks; ++r) th.emplace_back(body, r);
  body(0);
  for (auto& t : th) t.join();
  clk::time_point end = t0;
  for (const auto& t : last)
    if (t > end) end = t;
  *span_ns = ns_since(end);
  return err.load();
}
