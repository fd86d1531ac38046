// Request queue of the serving entry points (wgw_submit / wgw_poll / wgw_wait / wgw_cancel):
// descriptor checks, admission against a device-memory budget, merging, cancellation and the
// ticket life cycle.  Host C++ only (no CUDA), so that the same code runs in the library's
// worker and in a host test harness that feeds it a fake memory reading.
#pragma once

#include <chrono>
#include <cmath>
#include <cstdint>
#include <deque>
#include <functional>
#include <map>
#include <set>
#include <string>
#include <utility>
#include <vector>

namespace wgw {
namespace serve {

constexpr int kOk = 0, kErrArg = 1, kErrNomem = 2, kErrCancelled = 7;
constexpr int kKindChi0 = 0, kKindChibar0 = 1, kKindPdep = 2;
constexpr int kMaxFrequencies = 4096;

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int kind = kKindChi0;
  int n_pert = 0;
  std::vector<double> dV;        // 2 N_rho n_pert, copied at submission
  std::vector<double> omega;
  double* out = nullptr;
  Clock::time_point t_submit;
};

struct Done {
  int status = kOk;
  double latency_s = 0, queue_s = 0;
  int batch_requests = 0, batch_systems = 0;
  std::string msg;   // what failed, for a status other than kOk
};

// Checks a request descriptor before anything is copied: a known kind, at least one
// perturbation, 1..kMaxFrequencies finite frequencies >= 0, non-null buffers, and finite
// perturbation coefficients.  A PDEP request (n_pert = number of eigenpairs) takes no
// frequencies, and its start block dV may be null.  Returns kOk or kErrArg with the reason in *why.
inline int validate(int kind, const double* dV, int n_pert, const double* omega, int n_omega, const double* out,
                    long n_rho, std::string* why) {
  auto bad = [&](const char* m) { if (why) *why = m; return kErrArg; };
  if (kind != kKindChi0 && kind != kKindChibar0 && kind != kKindPdep) return bad("unknown request kind");
  if (n_pert < 1) return bad("need n_pert >= 1");
  if (kind == kKindPdep) {
    if (!out) return bad("null out");
    if (dV)
      for (size_t i = 0; i < 2 * (size_t)n_rho * n_pert; ++i)
        if (!std::isfinite(dV[i])) return bad("start block coefficients must be finite");
    return kOk;
  }
  if (n_omega < 1 || n_omega > kMaxFrequencies) return bad("need 1 <= n_omega <= 4096 frequencies");
  if (!dV || !omega || !out) return bad("null dV, omega or out");
  for (int k = 0; k < n_omega; ++k)
    if (!(omega[k] >= 0.0) || !std::isfinite(omega[k])) return bad("frequencies must be finite and >= 0");
  const size_t n = 2 * (size_t)n_rho * n_pert;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(dV[i])) return bad("perturbation coefficients must be finite");
  return kOk;
}

// The queue.  Not thread-safe by itself: the owner serialises calls (one mutex).
class Queue {
 public:
  uint64_t push(Request r) {
    r.ticket = next_++;
    const uint64_t t = r.ticket;
    queue_.push_back(std::move(r));
    return t;
  }

  bool empty() const { return queue_.empty(); }
  size_t queued() const { return queue_.size(); }

  // The next batch.  bytes_for(n_real, whole) is the device memory an apply of n_real real-in-r
  // perturbation parts (at most twice the perturbations) needs: with whole = false the least it
  // can run in (one perturbation per chunk, plus its inputs and outputs), with whole = true all
  // of them resident at once.  The head request is admitted when its least need fits `budget`;
  // if it does not, it waits while other work runs (device_busy) and is completed with
  // kErrNomem when the device is idle (it can never fit).  Requests rejected that way are
  // appended to *rejected.  Every later queued request of the head's kind and frequency set
  // joins, in submission order, while the whole batch stays resident within the budget.
  // Returns the batch (empty when nothing runs).
  std::vector<Request> take_batch(double budget, const std::function<double(int, bool)>& bytes_for, bool device_busy,
                                  std::vector<std::pair<uint64_t, Done>>* rejected) {
    std::vector<Request> batch;
    while (!queue_.empty()) {
      Request& head = queue_.front();
      if (bytes_for(2 * head.n_pert, false) <= budget) break;
      if (device_busy) return batch;
      Done d;
      d.status = kErrNomem;
      d.latency_s = d.queue_s = std::chrono::duration<double>(Clock::now() - head.t_submit).count();
      if (rejected) rejected->emplace_back(head.ticket, d);
      done_[head.ticket] = d;
      queue_.pop_front();
    }
    if (queue_.empty()) return batch;
    const int kind = queue_.front().kind;
    const std::vector<double> om = queue_.front().omega;
    int n_tot = 0;
    for (auto it = queue_.begin(); it != queue_.end();) {
      if (it->kind == kind && it->omega == om &&
          (batch.empty() || bytes_for(2 * (n_tot + it->n_pert), true) <= budget)) {
        n_tot += it->n_pert;
        running_.insert(it->ticket);
        batch.push_back(std::move(*it));
        it = queue_.erase(it);
      } else {
        ++it;
      }
    }
    return batch;
  }

  // The head request, moved out and marked running, if it satisfies `take`; false otherwise.
  template <typename F>
  bool take_head_if(F&& take, Request* out) {
    if (queue_.empty() || !take(queue_.front())) return false;
    *out = std::move(queue_.front());
    queue_.pop_front();
    running_.insert(out->ticket);
    return true;
  }
  const Request* head() const { return queue_.empty() ? nullptr : &queue_.front(); }

  // Cancels a request: a queued one is removed and completed with kErrCancelled at once; a
  // running one completes with kErrCancelled when its batch ends (its output is not written).
  // Returns kErrArg for an unknown or already finished ticket.
  int cancel(uint64_t ticket) {
    for (auto it = queue_.begin(); it != queue_.end(); ++it)
      if (it->ticket == ticket) {
        Done d;
        d.status = kErrCancelled;
        d.latency_s = d.queue_s = std::chrono::duration<double>(Clock::now() - it->t_submit).count();
        done_[ticket] = d;
        queue_.erase(it);
        return kOk;
      }
    if (running_.count(ticket)) {
      cancelled_.insert(ticket);
      return kOk;
    }
    return kErrArg;
  }

  bool cancelled(uint64_t ticket) const { return cancelled_.count(ticket) > 0; }

  // Completes the requests of a batch with `status` (kErrCancelled for the cancelled ones).
  void finish(const std::vector<Request>& batch, int status, Clock::time_point t_start, Clock::time_point t_end,
              int batch_systems, const std::string& msg = std::string()) {
    for (const Request& r : batch) {
      Done d;
      d.status = cancelled_.count(r.ticket) ? kErrCancelled : status;
      if (d.status != kOk) d.msg = d.status == kErrCancelled ? "request cancelled" : msg;
      d.latency_s = std::chrono::duration<double>(t_end - r.t_submit).count();
      d.queue_s = std::chrono::duration<double>(t_start - r.t_submit).count();
      d.batch_requests = (int)batch.size();
      d.batch_systems = batch_systems;
      done_[r.ticket] = d;
      running_.erase(r.ticket);
      cancelled_.erase(r.ticket);
    }
  }

  // Completes one running request (kErrCancelled if it was cancelled) with its own batch figures.
  void finish_one(const Request& r, int status, Clock::time_point t_start, Clock::time_point t_end, int batch_requests,
                  int batch_systems, const std::string& msg = std::string()) {
    Done d;
    d.status = cancelled_.count(r.ticket) ? kErrCancelled : status;
    if (d.status != kOk) d.msg = d.status == kErrCancelled ? "request cancelled" : msg;
    d.latency_s = std::chrono::duration<double>(t_end - r.t_submit).count();
    d.queue_s = std::chrono::duration<double>(t_start - r.t_submit).count();
    d.batch_requests = batch_requests;
    d.batch_systems = batch_systems;
    done_[r.ticket] = d;
    running_.erase(r.ticket);
    cancelled_.erase(r.ticket);
  }

  enum State { kUnknown = 0, kQueued, kRunning, kDone };
  State state(uint64_t ticket) const {
    if (done_.count(ticket)) return kDone;
    if (running_.count(ticket)) return kRunning;
    for (const Request& r : queue_)
      if (r.ticket == ticket) return kQueued;
    return kUnknown;
  }

  // Takes the result of a finished request (releasing the ticket); false if not finished.
  bool take_done(uint64_t ticket, Done* d) {
    auto it = done_.find(ticket);
    if (it == done_.end()) return false;
    if (d) *d = it->second;
    done_.erase(it);
    return true;
  }

 private:
  std::deque<Request> queue_;
  std::map<uint64_t, Done> done_;
  std::set<uint64_t> running_, cancelled_;
  uint64_t next_ = 1;
};

}  // namespace serve
}  // namespace wgw
