// Per-device one-time set-up (host code only, no CUDA headers).
//
// Kernel attributes such as the dynamic shared-memory limit belong to a device
// context, not to the process: a set-up that runs once per process leaves every
// other device without it.  once_for_device runs f() the first time it is called
// for each device index 0..63 (remembered as bits of `done`); for any other index
// it runs f() on every call.  Two threads racing on the same device may both run
// f(), so f must be idempotent.
#pragma once

#include <atomic>
#include <cstdint>

namespace stm {

template <typename F>
void once_for_device(std::atomic<uint64_t>& done, int dev, F&& f) {
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  f();
  if (bit) done.fetch_or(bit, std::memory_order_release);
}

}  // namespace stm
