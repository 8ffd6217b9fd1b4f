// Admission policy of the request server, as host logic only (no CUDA), so that it can be
// exercised on its own.  The caller holds the server's lock around every call.
//
// Requests wait per detector in submission order.  A detector has kSlots staging slots, so at
// most kSlots of its launch sets are in flight; the staged bytes of everything in flight stay
// within the budget (a request larger than the budget is admitted alone, when nothing else is
// in flight).  Only the head of a detector's queue can start: a head that does not fit keeps
// the detector's later requests waiting, so each detector sees its requests in submission
// order.  Among the admissible heads of a scheduler thread's detectors (detector d belongs to
// thread d mod T) the one with the smallest ticket starts.  An insert takes the inserts that
// directly follow it in its detector's queue into its launch set, up to merge_max points and
// within the budget, unless the detector may not merge (a sliding window evicts per batch).
//
// Req needs the fields id (ticket, increasing in submission order), det, op, dtype, n, bytes
// and merged (a std::vector<Req*>).
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <vector>

namespace ace {

template <typename Req>
struct Admission {
  static constexpr int kSlots = 2;        // staging slots per detector
  std::vector<std::deque<Req*>> waiting;  // per detector, in submission order
  std::vector<int64_t> npending;          // waiting requests per scheduler thread
  std::vector<int> inflight;              // launch sets in flight per detector
  size_t budget = 0, bytes_inflight = 0;
  int64_t merge_max = 65536;              // points of one coalesced insert
  uint64_t coalesced = 0;                 // requests admitted inside another's launch set

  void init(int ndet, int nthreads, size_t budget_bytes) {
    waiting.assign(static_cast<size_t>(ndet), std::deque<Req*>());
    npending.assign(static_cast<size_t>(nthreads), 0);
    inflight.assign(static_cast<size_t>(ndet), 0);
    budget = budget_bytes;
  }

  int nthreads() const { return static_cast<int>(npending.size()); }

  void submit(Req* r) {
    waiting[static_cast<size_t>(r->det)].push_back(r);
    npending[static_cast<size_t>(r->det % nthreads())] += 1;
  }

  // The request thread w starts next (with its merged inserts), taken off the queue, or
  // nullptr.  mergeable(det) says whether detector det's inserts may be coalesced; insert_op
  // is the insert operation's code.
  template <typename Mergeable>
  Req* pick(int w, int insert_op, Mergeable mergeable) {
    Req* r = nullptr;
    for (size_t d = static_cast<size_t>(w); d < waiting.size(); d += static_cast<size_t>(nthreads())) {
      if (waiting[d].empty() || inflight[d] >= kSlots) continue;
      Req* h = waiting[d].front();
      if (bytes_inflight != 0 && bytes_inflight + h->bytes > budget) continue;
      if (!r || h->id < r->id) r = h;
    }
    if (!r) return nullptr;
    std::deque<Req*>& q = waiting[static_cast<size_t>(r->det)];
    q.pop_front();
    size_t bytes = r->bytes;
    int64_t n = r->n;
    if (r->op == insert_op && mergeable(r->det)) {
      while (!q.empty()) {
        Req* o = q.front();
        if (o->op != insert_op || o->dtype != r->dtype || n + o->n > merge_max ||
            bytes_inflight + bytes + o->bytes > budget)
          break;
        r->merged.push_back(o);
        bytes += o->bytes;
        n += o->n;
        q.pop_front();
      }
    }
    npending[static_cast<size_t>(w)] -= 1 + static_cast<int64_t>(r->merged.size());
    coalesced += r->merged.size();
    return r;
  }

  // r (picked) is in flight: its slot and its bytes, and those of its merged inserts.
  void start(const Req* r) {
    inflight[static_cast<size_t>(r->det)] += 1;
    bytes_inflight += r->bytes;
    for (const Req* q : r->merged) bytes_inflight += q->bytes;
  }

  // r's launch set has completed (or could not be enqueued): its slot and bytes are free.
  void finish(const Req* r) {
    inflight[static_cast<size_t>(r->det)] -= 1;
    bytes_inflight -= r->bytes;
    for (const Req* q : r->merged) bytes_inflight -= q->bytes;
  }

  // Nothing waiting and nothing in flight.
  bool idle() const {
    for (int64_t v : npending)
      if (v) return false;
    for (int v : inflight)
      if (v) return false;
    return true;
  }
};

}  // namespace ace
