// Test-only host harness around the library's request queue (csrc/serve_sched.h): the same
// queue class the serving worker uses, driven with a fake device-memory reading so that
// admission, merging, cancellation and descriptor checks can be tested without a GPU.  Built
// only by tests/test_serve_host.py; not part of libwgw.
#include <cstdint>
#include <vector>

#include "serve_sched.h"

using wgw::serve::Done;
using wgw::serve::Queue;
using wgw::serve::Request;

namespace {
// Fake memory model: an apply of n_real real-in-r parts needs base + per_real * (n_real if
// resident as a whole, else 1) bytes.
struct Harness {
  Queue q;
  double base = 0, per_real = 0;
};
}  // namespace

extern "C" {

void* sh_new(double base, double per_real) {
  Harness* h = new Harness();
  h->base = base;
  h->per_real = per_real;
  return h;
}

void sh_free(void* p) { delete static_cast<Harness*>(p); }

int sh_validate(int kind, const double* dV, int n_pert, const double* omega, int n_omega, const double* out,
                long n_rho) {
  return wgw::serve::validate(kind, dV, n_pert, omega, n_omega, out, n_rho, nullptr);
}

uint64_t sh_push(void* p, int kind, int n_pert, const double* omega, int n_omega) {
  Request r;
  r.kind = kind;
  r.n_pert = n_pert;
  r.omega.assign(omega, omega + n_omega);
  r.t_submit = wgw::serve::Clock::now();
  return static_cast<Harness*>(p)->q.push(std::move(r));
}

// Takes one batch with the fake memory model and `budget`; writes the batch's tickets and the
// rejected tickets.  Returns the batch size.
int sh_take(void* p, double budget, int busy, uint64_t* batch, int n_max, uint64_t* rejected, int* n_rejected) {
  Harness* h = static_cast<Harness*>(p);
  std::vector<std::pair<uint64_t, Done>> rej;
  auto bytes = [&](int n_real, bool whole) { return h->base + h->per_real * (whole ? n_real : 1); };
  std::vector<Request> b = h->q.take_batch(budget, bytes, busy != 0, &rej);
  for (size_t k = 0; k < rej.size(); ++k) rejected[k] = rej[k].first;
  *n_rejected = (int)rej.size();
  const int n = (int)b.size();
  for (int k = 0; k < n && k < n_max; ++k) batch[k] = b[k].ticket;
  h->q.finish(b, 0, wgw::serve::Clock::now(), wgw::serve::Clock::now(), 0);
  return n;
}

// Takes one batch and leaves it running (not finished); returns its size.
int sh_take_running(void* p, double budget, uint64_t* batch, int n_max) {
  Harness* h = static_cast<Harness*>(p);
  auto bytes = [&](int n_real, bool whole) { return h->base + h->per_real * (whole ? n_real : 1); };
  std::vector<Request> b = h->q.take_batch(budget, bytes, false, nullptr);
  const int n = (int)b.size();
  for (int k = 0; k < n && k < n_max; ++k) batch[k] = b[k].ticket;
  static std::vector<Request> keep;
  keep = std::move(b);
  return n;
}

// Finishes the batch left running by sh_take_running with `status`.
void sh_finish_running(void* p, int status, const uint64_t* tickets, int n) {
  Harness* h = static_cast<Harness*>(p);
  std::vector<Request> b(n);
  for (int k = 0; k < n; ++k) b[k].ticket = tickets[k];
  h->q.finish(b, status, wgw::serve::Clock::now(), wgw::serve::Clock::now(), 0);
}

int sh_cancel(void* p, uint64_t t) { return static_cast<Harness*>(p)->q.cancel(t); }

int sh_state(void* p, uint64_t t) { return (int)static_cast<Harness*>(p)->q.state(t); }

// Status of a finished request (releasing its ticket), or -1 if it has not finished.
int sh_take_done(void* p, uint64_t t) {
  Done d;
  return static_cast<Harness*>(p)->q.take_done(t, &d) ? d.status : -1;
}

}  // extern "C"
