// Bounded wait on a device flag written by other blocks of the same launch (the batched
// launch's hand-over from hash blocks to query blocks, and from the block that derives a
// detector's threshold to its flag blocks).
#pragma once

#include "ace_internal.h"

namespace ace {

constexpr long long kFlagWait = 4000000000LL;  // about 2 s at 2 GHz

// Waits (one thread) until *flag >= want, bounded by `limit` SM cycles; on time-out it raises
// ACE_STATUS_TIMEOUT in st->status and gives up (the results it guards are then not to be
// used).  Returns whether the flag was reached.
__device__ __forceinline__ bool wait_at_least(const unsigned int* flag, unsigned int want, DevStats* st,
                                              long long limit = kFlagWait) {
  const long long t0 = clock64();
  bool ok = true;
  while (*reinterpret_cast<const volatile unsigned int*>(flag) < want) {
    if (clock64() - t0 > limit) {
      atomicOr(&st->status, static_cast<unsigned>(ACE_STATUS_TIMEOUT));
      ok = false;
      break;
    }
    __nanosleep(256);
  }
  __threadfence();
  return ok;
}

}  // namespace ace
