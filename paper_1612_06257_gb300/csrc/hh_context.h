// hh_context.h -- the hh_ctx object behind the C ABI (library-internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "hh_internal.h"

namespace hh {

// Device buffers of one chunk slot of the host-buffer path.
struct HostSlot {
  uint8_t* bytes = nullptr;
  size_t bytes_cap = 0;
  int64_t* offsets = nullptr;
  size_t offsets_cap = 0;  // elements
  uint64_t* keys = nullptr;
  size_t keys_cap = 0;     // elements
  uint64_t* out = nullptr;
  size_t out_cap = 0;      // elements
  cudaEvent_t staged = nullptr;   // inputs on the device
  cudaEvent_t hashed = nullptr;   // kernel done
  cudaEvent_t drained = nullptr;  // output copied back: slot reusable
};

// Fixed-length batches are tuned per length class:
// len <= 64, <= 256, <= 1024, <= 8192, larger.
constexpr int kFixedClasses = 5;
constexpr int64_t kFixedClassMax[kFixedClasses - 1] = {64, 256, 1024, 8192};

inline int fixed_class(int64_t len) {
  int c = 0;
  while (c < kFixedClasses - 1 && len > kFixedClassMax[c]) ++c;
  return c;
}

// The choices the autotuner makes (defaults: measured on GB300).
struct TuneTable {
  StagedShape fixed[kFixedClasses] = {{128, 2, 2}, {128, 2, 2}, {128, 2, 2}, {128, 2, 2},
                                      {256, 2, 1}};
  StagedShape ragged{256, 2};  // warp-tile kernel
  int huge_bucket = kHugeBucket;  // messages in this bucket and above run two threads each
  int solo_per_sm = kSoloPerSm;   // up to this many huge messages per SM: one warp each
  int solo_shared = 1;            // 1: solo tiles also beside other launches in flight
  int fixed_pair = 1;             // small fixed batches: 1 two threads per message, 0 one
};

// Read a table written by hh_tune_save; false (t unchanged) on a bad file.
bool load_tune_table(const char* path, TuneTable& t);

// Makes `dev` the current device for the guard's lifetime.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace hh

struct hh_ctx {
  int device = 0;
  int num_sms = 0;
  int kernel = HH_KERNEL_AUTO;
  int* d_err = nullptr;
  unsigned long long* d_next_tile = nullptr;  // [4]: the work queue's counters
  int* d_use_perm = nullptr;
  long long* d_huge = nullptr;
  uint32_t* d_hist = nullptr;
  uint32_t* d_cursor = nullptr;
  int32_t* d_perm = nullptr;
  int64_t perm_cap = 0;
  hh::TuneTable tune;
  std::string tune_report;  // per-candidate times of the last hh_autotune (comment lines)
  hh::StagedShape shape_bulk{256, 2};  // per-thread bulk-copy kernel
  int last_launches = 0;
  bool tuning = false;  // hh_autotune is timing shapes: no small-batch override
  uint64_t wait_limit_ns = hh::kWaitLimitNs;  // limit of one wait for an asynchronous copy
  // Host-buffer path.
  cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
  hh::HostSlot slots[2];
};
