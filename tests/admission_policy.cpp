// Self-checking scenarios for the request server's admission policy (admission.h), host code
// only: per-detector order, the two staging slots, the memory budget, coalescing of
// consecutive inserts, the split of detectors among scheduler threads, and a randomised run
// whose invariants are checked at every step.  Prints "ok <checks>" and exits 0, or names the
// first failed check and exits 1.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "admission.h"

namespace {

constexpr int kInsert = 1, kScore = 2;  // two operation codes, as the server's

struct Req {
  uint64_t id = 0;
  int det = 0, op = 0, dtype = 0;
  int64_t n = 0;
  size_t bytes = 0;
  std::vector<Req*> merged;
};

int g_checks = 0;

void check(bool ok, const char* what, int line) {
  ++g_checks;
  if (!ok) {
    std::printf("FAILED line %d: %s\n", line, what);
    std::exit(1);
  }
}
#define CHECK(c) check((c), #c, __LINE__)

struct Pool {
  std::vector<Req*> all;
  uint64_t next = 1;
  Req* make(int det, int op, int64_t n, size_t bytes, int dtype = 0) {
    Req* r = new Req();
    r->id = next++;
    r->det = det;
    r->op = op;
    r->n = n;
    r->bytes = bytes;
    r->dtype = dtype;
    all.push_back(r);
    return r;
  }
  ~Pool() {
    for (Req* r : all) delete r;
  }
};

auto always = [](int) { return true; };

void order_and_slots() {
  ace::Admission<Req> a;
  a.init(2, 1, 1 << 20);
  Pool p;
  Req* A = p.make(0, kInsert, 10, 100);
  Req* B = p.make(0, kScore, 10, 100);
  Req* C = p.make(0, kInsert, 10, 100);
  for (Req* r : {A, B, C}) a.submit(r);
  Req* r = a.pick(0, kInsert, always);
  CHECK(r == A && A->merged.empty());  // a score between two inserts stops the merge
  a.start(r);
  r = a.pick(0, kInsert, always);
  CHECK(r == B);
  a.start(r);
  CHECK(a.pick(0, kInsert, always) == nullptr);  // both slots of detector 0 are in flight
  a.finish(A);
  r = a.pick(0, kInsert, always);
  CHECK(r == C);
  a.start(r);
  a.finish(B);
  a.finish(C);
  CHECK(a.idle() && a.bytes_inflight == 0);
}

void coalescing() {
  ace::Admission<Req> a;
  a.init(3, 1, 1 << 20);
  Pool p;
  std::vector<Req*> ins;
  for (int i = 0; i < 5; ++i) ins.push_back(p.make(1, kInsert, 100, 1000));
  Req* other = p.make(2, kScore, 5, 50);  // another detector's request does not stop the merge
  Req* more = p.make(1, kInsert, 100, 1000);
  for (Req* r : ins) a.submit(r);
  a.submit(other);
  a.submit(more);
  Req* r = a.pick(0, kInsert, always);
  CHECK(r == ins[0] && r->merged.size() == 5 && r->merged[4] == more);
  CHECK(a.coalesced == 5 && a.npending[0] == 1);
  a.start(r);
  CHECK(a.bytes_inflight == 6000);
  Req* s = a.pick(0, kInsert, always);
  CHECK(s == other);
  a.start(s);
  a.finish(r);
  a.finish(s);
  CHECK(a.idle() && a.bytes_inflight == 0);

  // the merged size stays within merge_max; another dtype and a non-mergeable detector stop it
  ace::Admission<Req> b;
  b.init(2, 1, 1 << 30);
  Pool q;
  Req* x = q.make(0, kInsert, 40000, 10);
  Req* y = q.make(0, kInsert, 30000, 10);
  Req* z = q.make(0, kInsert, 20000, 10);
  b.submit(x);
  b.submit(y);
  b.submit(z);
  r = b.pick(0, kInsert, always);
  CHECK(r == x && r->merged.empty());  // 40000 + 30000 > 65536
  b.start(r);
  r = b.pick(0, kInsert, always);
  CHECK(r == y && r->merged.size() == 1 && r->merged[0] == z);  // 30000 + 20000 fits
  Req* u = q.make(1, kInsert, 10, 10, 0);
  Req* v = q.make(1, kInsert, 10, 10, 1);  // other input type
  b.submit(u);
  b.submit(v);
  r = b.pick(0, kInsert, always);
  CHECK(r == u && r->merged.empty());
  Req* w1 = q.make(1, kInsert, 10, 10);
  Req* w2 = q.make(1, kInsert, 10, 10);
  b.submit(w1);
  b.submit(w2);
  b.start(r);
  b.finish(r);
  r = b.pick(0, kInsert, [](int d) { return d != 1; });  // detector 1 keeps a sliding window
  CHECK(r == v && r->merged.empty());
  b.start(r);
  r = b.pick(0, kInsert, [](int d) { return d != 1; });
  CHECK(r == w1 && r->merged.empty());
}

void budget() {
  ace::Admission<Req> a;
  a.init(4, 1, 1000);
  Pool p;
  Req* big = p.make(0, kScore, 1, 600);
  Req* held = p.make(1, kScore, 1, 500);
  Req* later = p.make(1, kScore, 1, 10);  // behind its detector's head
  Req* fits = p.make(2, kScore, 1, 300);
  for (Req* r : {big, held, later, fits}) a.submit(r);
  Req* r = a.pick(0, kInsert, always);
  CHECK(r == big);
  a.start(r);
  r = a.pick(0, kInsert, always);
  CHECK(r == fits);  // detector 1's head does not fit and keeps `later` behind it
  a.start(r);
  CHECK(a.pick(0, kInsert, always) == nullptr);
  a.finish(big);
  r = a.pick(0, kInsert, always);
  CHECK(r == held);
  a.start(r);
  a.finish(fits);
  a.finish(held);
  // a request larger than the budget starts alone, once nothing else is in flight
  Req* huge = p.make(3, kScore, 1, 5000);
  a.submit(huge);
  r = a.pick(0, kInsert, always);
  CHECK(r == later);
  a.start(r);
  CHECK(a.pick(0, kInsert, always) == nullptr);
  a.finish(later);
  r = a.pick(0, kInsert, always);
  CHECK(r == huge);
  a.start(r);
  a.finish(r);
  CHECK(a.idle());
}

void earliest_and_threads() {
  ace::Admission<Req> a;
  a.init(4, 2, 1 << 20);
  Pool p;
  Req* d0 = p.make(0, kScore, 1, 1);
  Req* d1 = p.make(1, kScore, 1, 1);
  Req* d2 = p.make(2, kScore, 1, 1);
  Req* d3 = p.make(3, kScore, 1, 1);
  for (Req* r : {d0, d1, d2, d3}) a.submit(r);
  CHECK(a.npending[0] == 2 && a.npending[1] == 2);
  Req* r = a.pick(1, kInsert, always);  // thread 1 owns detectors 1 and 3
  CHECK(r == d1);
  r = a.pick(1, kInsert, always);
  CHECK(r == d3);
  CHECK(a.pick(1, kInsert, always) == nullptr);
  r = a.pick(0, kInsert, always);
  CHECK(r == d0);
  r = a.pick(0, kInsert, always);
  CHECK(r == d2);
  CHECK(a.npending[0] == 0 && a.npending[1] == 0);
}

// Random submissions and completions on 6 detectors, 2 threads, a tight budget: at every step
// at most two launch sets per detector are in flight, the staged bytes fit the budget unless
// one set alone is in flight, each detector's requests start in submission order, and every
// request starts once the rest complete.
void randomised() {
  std::mt19937_64 rng(7);
  const int ndet = 6, nthr = 2;
  ace::Admission<Req> a;
  a.init(ndet, nthr, 20000);
  Pool p;
  std::vector<std::vector<uint64_t>> submitted(ndet), started(ndet);
  std::vector<Req*> flight;
  int total = 0, done = 0;
  for (int step = 0; step < 20000; ++step) {
    const int act = static_cast<int>(rng() % 3);
    if (act == 0 && total < 4000) {
      const int det = static_cast<int>(rng() % ndet);
      const int op = (rng() % 2) ? kInsert : kScore;
      const int64_t n = 1 + static_cast<int64_t>(rng() % 30000);
      Req* r = p.make(det, op, n, static_cast<size_t>(n) / 4 + (rng() % 50 == 0 ? 30000 : 0), 0);
      a.submit(r);
      submitted[det].push_back(r->id);
      ++total;
    } else if (act == 1) {
      Req* r = a.pick(static_cast<int>(rng() % nthr), kInsert, [](int d) { return d != 5; });
      if (r) {
        CHECK(a.inflight[static_cast<size_t>(r->det)] < 2);
        size_t b = r->bytes;
        int64_t n = r->n;
        for (Req* q : r->merged) {
          b += q->bytes;
          n += q->n;
          CHECK(q->det == r->det && q->op == kInsert && r->op == kInsert && r->det != 5);
        }
        CHECK(r->merged.empty() || n <= a.merge_max);
        CHECK(a.bytes_inflight == 0 || a.bytes_inflight + b <= a.budget);
        a.start(r);
        started[r->det].push_back(r->id);
        for (Req* q : r->merged) started[r->det].push_back(q->id);
        flight.push_back(r);
      }
    } else if (!flight.empty()) {
      const size_t k = static_cast<size_t>(rng() % flight.size());
      a.finish(flight[k]);
      done += 1 + static_cast<int>(flight[k]->merged.size());
      flight.erase(flight.begin() + static_cast<long>(k));
    }
    for (int d = 0; d < ndet; ++d) {
      const int f = a.inflight[static_cast<size_t>(d)];
      CHECK(f >= 0 && f <= 2);
    }
  }
  // drain: complete everything, starting what remains
  for (;;) {
    Req* r = nullptr;
    for (int w = 0; w < nthr && !r; ++w) r = a.pick(w, kInsert, [](int d) { return d != 5; });
    if (r) {
      a.start(r);
      started[r->det].push_back(r->id);
      for (Req* q : r->merged) started[r->det].push_back(q->id);
      flight.push_back(r);
      continue;
    }
    if (flight.empty()) break;
    a.finish(flight.back());
    done += 1 + static_cast<int>(flight.back()->merged.size());
    flight.pop_back();
  }
  CHECK(a.idle() && a.bytes_inflight == 0 && done == total);
  for (int d = 0; d < ndet; ++d) CHECK(started[d] == submitted[d]);
  CHECK(a.coalesced > 0);
}

}  // namespace

int main() {
  order_and_slots();
  coalescing();
  budget();
  earliest_and_threads();
  randomised();
  std::printf("ok %d\n", g_checks);
  return 0;
}
