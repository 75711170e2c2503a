// hh_tune.cu -- the autotuner and its tuning table.
//
// hh_autotune times the candidate kernel shapes on synthetic batches in
// device memory and keeps the fastest per length regime:
//   * fixed-length batches, per length class (<= 64, <= 256, <= 1024,
//     <= 8192 bytes, larger; timed at 64, 256, 1024, 4096, 65536): the TMA
//     kernel's window, pipeline depth and messages per thread;
//   * ragged batches (log-uniform lengths in [0, 65536]): the warp-tile
//     kernel's window and pipeline depth;
//   * long messages (log-uniform 64 KiB - 4 MiB after short ones): the length
//     from which a message runs two threads per message, or never;
//   * 8 long messages per SM: up to how many long messages per SM each gets
//     a warp of its own (solo tiles) instead of sharing one (pair tiles).
// The table can be written with hh_tune_save and read back by hh_init.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hh.h"
#include "hh_context.h"
#include "hh_internal.h"

namespace {

// splitmix64 (Vigna) of a counter: the synthetic bytes of the tuning batches.
__global__ void fill_kernel(uint64_t* p, int64_t words, uint64_t seed) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < words;
       i += stride) {
    uint64_t z = seed + static_cast<uint64_t>(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    p[i] = z ^ (z >> 31);
  }
}

struct Buffers {
  uint8_t* bytes = nullptr;
  int64_t* offsets = nullptr;
  uint64_t* keys = nullptr;
  uint64_t* out = nullptr;
  ~Buffers() {
    cudaFree(bytes);
    cudaFree(offsets);
    cudaFree(keys);
    cudaFree(out);
  }
};

// Milliseconds per call of `call`, averaged over `reps` calls between two
// events on `s`; a huge value if a call fails.
template <class F>
float time_calls(F call, cudaStream_t s, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  bool ok = true;
  for (int i = 0; i < reps; ++i) ok = ok && call() == HH_OK;
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ok ? ms / reps : 1e30f;
}

// Index of the fastest of `count` candidates.  apply(i) installs candidate i
// and call() runs the batch once.  Every candidate is warmed up, the
// repetition count is set so that one sample takes about 5 ms, and the
// candidates are timed in kRounds interleaved rounds (so clock changes hit
// all of them alike); each keeps its best sample.
template <class A, class F>
int fastest(int count, A apply, F call, cudaStream_t s, std::vector<float>& best) {
  constexpr int kRounds = 4;
  best.assign(count, 1e30f);
  int reps = 1;
  for (int i = 0; i < count; ++i) {
    apply(i);
    const float ms = time_calls(call, s, 1);
    if (ms < 1e29f && ms > 0) {
      const int r = static_cast<int>(5.0f / ms);
      reps = std::max(reps, std::min(r, 200));
    }
  }
  for (int round = 0; round < kRounds; ++round)
    for (int i = 0; i < count; ++i) {
      apply(i);
      best[i] = std::min(best[i], time_calls(call, s, reps));
    }
  int pick = 0;
  for (int i = 1; i < count; ++i)
    if (best[i] < best[pick]) pick = i;
  return best[pick] < 1e29f ? pick : -1;
}

// One comment line of the tuning report: each candidate's best time.
template <class L>
void report_line(std::string& r, const char* what, const std::vector<float>& ms, L label) {
  r += "# ";
  r += what;
  char cell[96];
  for (size_t i = 0; i < ms.size(); ++i) {
    std::snprintf(cell, sizeof(cell), " %s=%.4gms", label(static_cast<int>(i)).c_str(), ms[i]);
    r += cell;
  }
  r += "\n";
}

std::string shape_label(const hh::StagedShape& sh) {
  char t[48];
  std::snprintf(t, sizeof(t), "%d/%d/%d", sh.window, sh.stages, sh.msgs);
  return t;
}

uint64_t next_random(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#define HH_LIST(W_, N_, M_) hh::StagedShape{W_, N_, M_},
const hh::StagedShape kFixedCandidates[] = {HH_FIXED_SHAPES(HH_LIST)};
#undef HH_LIST
#define HH_LIST(W_, N_) hh::StagedShape{W_, N_, 1},
const hh::StagedShape kRaggedCandidates[] = {HH_RAGGED_SHAPES(HH_LIST)};
#undef HH_LIST

}  // namespace

namespace hh {
bool set_tune_scalar(TuneTable& t, const char* name, int value);
}

extern "C" {

int hh_autotune(hh_ctx* ctx, int64_t max_device_bytes) {
  if (ctx == nullptr || max_device_bytes < (int64_t(64) << 20)) return HH_ERR_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return HH_ERR_CUDA;
  const int saved_kernel = ctx->kernel;
  ctx->kernel = HH_KERNEL_AUTO;
  ctx->tuning = true;
  const int64_t budget = max_device_bytes & ~int64_t(4095);
  const int64_t max_msgs = int64_t(1) << 22;
  Buffers buf;
  cudaStream_t s = nullptr;
  int status = HH_OK;
  std::vector<float> ms;
  std::string report;
  char what[96];
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&buf.bytes, budget) != cudaSuccess ||
      cudaMalloc(&buf.offsets, sizeof(int64_t) * (max_msgs + 1)) != cudaSuccess ||
      cudaMalloc(&buf.keys, sizeof(uint64_t) * 4) != cudaSuccess ||
      cudaMalloc(&buf.out, sizeof(uint64_t) * max_msgs * 4) != cudaSuccess) {
    status = HH_ERR_NO_MEMORY;
  }
  if (status == HH_OK) {
    fill_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(reinterpret_cast<uint64_t*>(buf.bytes),
                                                  budget / 8, 0x1234u);
    fill_kernel<<<1, 32, 0, s>>>(buf.keys, 4, 0x5678u);
    if (cudaStreamSynchronize(s) != cudaSuccess) status = HH_ERR_CUDA;
  }
  status = status == HH_OK ? hh_reserve(ctx, max_msgs) : status;

  // Fixed-length classes.
  const int64_t class_len[hh::kFixedClasses] = {64, 256, 1024, 4096, 65536};
  const int n_fixed = static_cast<int>(sizeof(kFixedCandidates) / sizeof(kFixedCandidates[0]));
  for (int c = 0; status == HH_OK && c < hh::kFixedClasses; ++c) {
    const int64_t len = class_len[c];
    const int64_t n = std::min(budget / len, max_msgs);
    const hh::StagedShape keep = ctx->tune.fixed[c];
    const int pick = fastest(
        n_fixed, [&](int i) { ctx->tune.fixed[c] = kFixedCandidates[i]; },
        [&] { return hh_hash_fixed(ctx, 64, buf.keys, HH_KEY_SHARED, buf.bytes, len, n, buf.out, s); },
        s, ms);
    std::snprintf(what, sizeof(what), "fixed %d (%lld x %lld B):", c, static_cast<long long>(n),
                  static_cast<long long>(len));
    report_line(report, what, ms, [](int i) { return shape_label(kFixedCandidates[i]); });
    ctx->tune.fixed[c] = pick < 0 ? keep : kFixedCandidates[pick];
    if (pick < 0) status = HH_ERR_CUDA;
  }

  // Ragged: log-uniform lengths in [0, 65536] filling most of the budget.
  std::vector<int64_t> off;
  if (status == HH_OK) {
    uint64_t state = 42;
    off.push_back(0);
    const double lmax = 65537.0;
    while (static_cast<int64_t>(off.size()) <= max_msgs) {
      const double u = (next_random(state) >> 11) * (1.0 / 9007199254740992.0);
      int64_t len = static_cast<int64_t>(std::exp(u * std::log(lmax))) - 1;
      if (len < 0) len = 0;
      if (off.back() + len > budget) break;
      off.push_back(off.back() + len);
    }
    const int64_t n = static_cast<int64_t>(off.size()) - 1;
    if (cudaMemcpy(buf.offsets, off.data(), sizeof(int64_t) * off.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      status = HH_ERR_CUDA;
    const hh::StagedShape keep = ctx->tune.ragged;
    const int n_ragged =
        static_cast<int>(sizeof(kRaggedCandidates) / sizeof(kRaggedCandidates[0]));
    const int pick =
        status != HH_OK
            ? -1
            : fastest(
                  n_ragged, [&](int i) { ctx->tune.ragged = kRaggedCandidates[i]; },
                  [&] {
                    return hh_hash64_batch(ctx, buf.keys, HH_KEY_SHARED, buf.bytes, buf.offsets,
                                           n, buf.out, s);
                  },
                  s, ms);
    std::snprintf(what, sizeof(what), "ragged (%lld messages, %lld B):", static_cast<long long>(n),
                  static_cast<long long>(off.back()));
    report_line(report, what, ms, [](int i) { return shape_label(kRaggedCandidates[i]); });
    ctx->tune.ragged = pick < 0 ? keep : kRaggedCandidates[pick];
    if (pick < 0) status = HH_ERR_CUDA;
  }

  // Pair tiles: lengths log-uniform in [64 KiB, 4 MiB] filling half the
  // budget, after 4096 messages of 40 bytes.  Candidates: pairs from
  // 128 KiB, 256 KiB, 512 KiB or 1 MiB up, or never.
  if (status == HH_OK) {
    uint64_t state = 7;
    off.assign(1, 0);
    for (int i = 0; i < 4096; ++i) off.push_back(off.back() + 40);
    const double lo = std::log(65536.0), hi = std::log(4194304.0);
    while (static_cast<int64_t>(off.size()) <= max_msgs) {
      const double u = (next_random(state) >> 11) * (1.0 / 9007199254740992.0);
      const int64_t len = static_cast<int64_t>(std::exp(lo + u * (hi - lo)));
      if (off.back() + len > budget / 2) break;
      off.push_back(off.back() + len);
    }
    const int64_t n = static_cast<int64_t>(off.size()) - 1;
    if (cudaMemcpy(buf.offsets, off.data(), sizeof(int64_t) * off.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      status = HH_ERR_CUDA;
    const int candidates[5] = {hh::bucket_of_packets(int64_t(128) << 10 >> 5),
                               hh::bucket_of_packets(int64_t(256) << 10 >> 5),
                               hh::bucket_of_packets(int64_t(512) << 10 >> 5),
                               hh::bucket_of_packets(int64_t(1024) << 10 >> 5), hh::kBuckets};
    const int keep = ctx->tune.huge_bucket;
    const int pick =
        status != HH_OK
            ? -1
            : fastest(
                  5, [&](int i) { ctx->tune.huge_bucket = candidates[i]; },
                  [&] {
                    return hh_hash64_batch(ctx, buf.keys, HH_KEY_SHARED, buf.bytes, buf.offsets,
                                           n, buf.out, s);
                  },
                  s, ms);
    std::snprintf(what, sizeof(what), "huge_bucket (%lld messages, %lld B):",
                  static_cast<long long>(n), static_cast<long long>(off.back()));
    report_line(report, what, ms, [&](int i) { return std::to_string(candidates[i]); });
    ctx->tune.huge_bucket = pick < 0 ? keep : candidates[pick];
    if (pick < 0) status = HH_ERR_CUDA;
  }

  // Solo tiles: 8 huge messages per SM (log-uniform [128 KiB, 2 MiB]) after
  // 4096 short ones; the candidates put the solo/pair boundary at 0 (pairs
  // only), 1, 2, 4 or 8 huge messages per SM.
  if (status == HH_OK) {
    uint64_t state = 11;
    off.assign(1, 0);
    for (int i = 0; i < 4096; ++i) off.push_back(off.back() + 40);
    const double lo = std::log(131072.0), hi = std::log(2097152.0);
    for (int i = 0; i < 8 * ctx->num_sms; ++i) {
      const double u = (next_random(state) >> 11) * (1.0 / 9007199254740992.0);
      const int64_t len = static_cast<int64_t>(std::exp(lo + u * (hi - lo)));
      if (off.back() + len > budget) break;
      off.push_back(off.back() + len);
    }
    const int64_t n = static_cast<int64_t>(off.size()) - 1;
    if (cudaMemcpy(buf.offsets, off.data(), sizeof(int64_t) * off.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      status = HH_ERR_CUDA;
    const int candidates[5] = {0, 1, 2, 4, 8};
    const int keep = ctx->tune.solo_per_sm;
    const int pick =
        status != HH_OK
            ? -1
            : fastest(
                  5, [&](int i) { ctx->tune.solo_per_sm = candidates[i]; },
                  [&] {
                    return hh_hash64_batch(ctx, buf.keys, HH_KEY_SHARED, buf.bytes, buf.offsets,
                                           n, buf.out, s);
                  },
                  s, ms);
    std::snprintf(what, sizeof(what), "solo_per_sm (%lld messages, %lld B):",
                  static_cast<long long>(n), static_cast<long long>(off.back()));
    report_line(report, what, ms, [&](int i) { return std::to_string(candidates[i]); });
    ctx->tune.solo_per_sm = pick < 0 ? keep : candidates[pick];
    if (pick < 0) status = HH_ERR_CUDA;
  }

  if (status == HH_OK && cudaStreamSynchronize(s) != cudaSuccess) status = HH_ERR_CUDA;
  if (s) cudaStreamDestroy(s);
  ctx->tune_report = status == HH_OK ? report : std::string();
  ctx->kernel = saved_kernel;
  ctx->tuning = false;
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return status;
}

int hh_tune_describe(hh_ctx* ctx, char* buf, int64_t buf_len) {
  if (ctx == nullptr || buf == nullptr || buf_len <= 0) return HH_ERR_INVALID_ARG;
  std::string text = "# libhh tuning table v1\n";
  char line[128];
  for (int c = 0; c < hh::kFixedClasses; ++c) {
    const hh::StagedShape& f = ctx->tune.fixed[c];
    std::snprintf(line, sizeof(line), "fixed %d %d %d %d\n", c, f.window, f.stages, f.msgs);
    text += line;
  }
  std::snprintf(line, sizeof(line), "ragged %d %d\n", ctx->tune.ragged.window,
                ctx->tune.ragged.stages);
  text += line;
  std::snprintf(line, sizeof(line), "huge_bucket %d\n", ctx->tune.huge_bucket);
  text += line;
  std::snprintf(line, sizeof(line), "solo_per_sm %d\n", ctx->tune.solo_per_sm);
  text += line;
  std::snprintf(line, sizeof(line), "solo_shared %d\n", ctx->tune.solo_shared);
  text += line;
  std::snprintf(line, sizeof(line), "fixed_pair %d\n", ctx->tune.fixed_pair);
  text += line;
  text += ctx->tune_report;
  if (static_cast<int64_t>(text.size()) + 1 > buf_len) return HH_ERR_TOO_LARGE;
  std::memcpy(buf, text.c_str(), text.size() + 1);
  return HH_OK;
}

int hh_set_tune_param(hh_ctx* ctx, const char* name, int value) {
  if (ctx == nullptr || name == nullptr) return HH_ERR_INVALID_ARG;
  if (std::strcmp(name, "wait_limit_ns") == 0) {
    // A property of the context, not of the tuning table (never saved).
    if (value < 0) return HH_ERR_INVALID_ARG;
    ctx->wait_limit_ns = static_cast<uint64_t>(value);
    return HH_OK;
  }
  return hh::set_tune_scalar(ctx->tune, name, value) ? HH_OK : HH_ERR_INVALID_ARG;
}

int hh_tune_save(hh_ctx* ctx, const char* path) {
  if (ctx == nullptr || path == nullptr) return HH_ERR_INVALID_ARG;
  char text[8192];
  const int st = hh_tune_describe(ctx, text, sizeof(text));
  if (st != HH_OK) return st;
  FILE* f = std::fopen(path, "w");
  if (f == nullptr) return HH_ERR_INVALID_ARG;
  const bool ok = std::fputs(text, f) >= 0;
  return (std::fclose(f) == 0 && ok) ? HH_OK : HH_ERR_INVALID_ARG;
}

}  // extern "C"

namespace hh {

// Set one scalar entry of a tuning table; false for an unknown name or a
// value out of range.
bool set_tune_scalar(TuneTable& t, const char* name, int value) {
  if (std::strcmp(name, "huge_bucket") == 0) {
    if (value < 0 || value > kBuckets) return false;
    t.huge_bucket = value;
  } else if (std::strcmp(name, "solo_per_sm") == 0) {
    if (value < 0 || value > 64) return false;
    t.solo_per_sm = value;
  } else if (std::strcmp(name, "solo_shared") == 0) {
    if (value != 0 && value != 1) return false;
    t.solo_shared = value;
  } else if (std::strcmp(name, "fixed_pair") == 0) {
    if (value != 0 && value != 1) return false;
    t.fixed_pair = value;
  } else {
    return false;
  }
  return true;
}

// Parse a table written by hh_tune_save into `t`; false on any bad line.
bool load_tune_table(const char* path, TuneTable& t) {
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) return false;
  TuneTable parsed = t;
  char line[256];
  bool ok = true;
  while (ok && std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int c, w, n, m;
    if (std::sscanf(line, "fixed %d %d %d %d", &c, &w, &n, &m) == 4) {
      const StagedShape sh{w, n, m};
      ok = c >= 0 && c < kFixedClasses && fixed_shape_valid(sh);
      if (ok) parsed.fixed[c] = sh;
    } else if (std::sscanf(line, "ragged %d %d", &w, &n) == 2) {
      const StagedShape sh{w, n, 1};
      ok = ragged_shape_valid(sh);
      if (ok) parsed.ragged = sh;
    } else {
      char name[32];
      ok = std::sscanf(line, "%31s %d", name, &c) == 2 && set_tune_scalar(parsed, name, c);
    }
  }
  std::fclose(f);
  if (ok) t = parsed;
  return ok;
}

}  // namespace hh
