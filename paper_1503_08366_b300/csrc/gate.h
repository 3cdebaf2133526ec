// Host-side turn-taking between two kinds of device work (no CUDA calls; compiled into the
// server and, on its own, into a CPU test).
#pragma once
#include <condition_variable>
#include <cstdint>
#include <mutex>

namespace pogs {

// Turns on the device between batched steps and large solves.  When the persistent batched
// kernel and the single-problem kernels shared the SMs, both ran far below their rates alone:
// the batched CTAs stay resident for a whole step, and the single-problem kernels are sized
// to whole waves of the device, so each fragments the other.  So a step holds the device alone
// (writer), large solves hold it together (readers), and the two alternate: every large solve
// that waited through a step enters before the next step starts (a phase-fair reader-writer
// gate; host side only, no device synchronisation).
struct GpuGate {
  std::mutex mu;
  std::condition_variable cv;
  int readers = 0;         // large solves holding the device
  int rwait = 0;           // large solves waiting
  int rpass = 0;           // waiting solves that enter before the next step
  int wwait = 0;           // steps waiting
  bool writer = false;     // a step holds the device
  uint64_t steps = 0;      // steps finished

  void read_lock() {
    std::unique_lock<std::mutex> lk(mu);
    const uint64_t seen = steps;
    ++rwait;
    cv.wait(lk, [&] { return !writer && (wwait == 0 || steps != seen); });
    --rwait;
    if (steps != seen && rpass > 0) --rpass;
    ++readers;
  }
  void read_unlock() {
    std::lock_guard<std::mutex> lk(mu);
    if (--readers == 0) cv.notify_all();
  }
  void write_lock() {
    std::unique_lock<std::mutex> lk(mu);
    ++wwait;
    cv.wait(lk, [&] { return !writer && readers == 0 && rpass == 0; });
    --wwait;
    writer = true;
  }
  void write_unlock() {
    std::lock_guard<std::mutex> lk(mu);
    writer = false;
    ++steps;
    rpass = rwait;
    cv.notify_all();
  }
};

}  // namespace pogs
