// hh_kernels.cu -- HighwayHash batch kernels for sm_103a.
//
// Two mappings, both one thread per message (the 1024-bit state stays in 32
// registers; Update has no cross-message dependency):
//
//  * naive_kernel: each thread reads its own message straight from global
//    memory.  Neighbouring threads read addresses a whole message apart, so
//    every load instruction touches 32 different cache lines.  Kept as the
//    plain baseline.
//
//  * staged_kernel: a CTA of 128 threads owns a tile of 128 messages.  For
//    each pipeline step every thread issues one bulk asynchronous copy
//    (cp.async.bulk, completing on an mbarrier) of the next W bytes of its
//    message into its own shared-memory row; NST buffers keep NST-1 steps in
//    flight while the thread hashes the previous step from shared memory.
//    The copies are 16-byte aligned supersets of each window, so a message at
//    any byte offset is realigned in registers with one PRMT per word; when
//    every message is 16-byte aligned a variant reads packets with 128-bit
//    shared loads instead.  Tiles are taken from a work queue in
//    length-descending order (longest first) when a length sort ran.
#include <cuda_runtime.h>

#include <cstdint>

#include "hh_batch.cuh"
#include "hh_device.cuh"
#include "hh_internal.h"
#include "hh_ptx.cuh"

namespace hh {
namespace {

// ------------------------------------------------------------ shared helpers

__device__ __forceinline__ void load_key(const Batch& b, int64_t m, uint64_t key[4]) {
  const uint64_t* k = key_of(b, m);
#pragma unroll
  for (int i = 0; i < 4; ++i) key[i] = __ldg(k + i);
}

__device__ __forceinline__ void store_digest(const Batch& b, int64_t m, const State& s, bool bad) {
  uint64_t h[4];
  digest(s, h);
  if (bad) h[0] = h[1] = h[2] = h[3] = 0;
  uint64_t* o = b.out + m * b.words;
  o[0] = h[0];
  if (b.words >= 2) o[1] = h[1];
  if (b.words == 4) {
    o[2] = h[2];
    o[3] = h[3];
  }
}

// 32 bytes at any address, byte by byte, as eight little-endian words.
__device__ __forceinline__ void load_packet_bytes(const uint8_t* p, uint32_t w[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    w[j] = static_cast<uint32_t>(p[4 * j]) | (static_cast<uint32_t>(p[4 * j + 1]) << 8) |
           (static_cast<uint32_t>(p[4 * j + 2]) << 16) | (static_cast<uint32_t>(p[4 * j + 3]) << 24);
  }
}

// ----------------------------------------------------------------- naive path

__global__ void __launch_bounds__(256) naive_kernel(Batch b) {
  resolve_count(b);
  const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= b.n) return;
  int64_t start, len;
  int bad;
  message_bounds(b, m, start, len, bad);
  if (bad) record_error(b.err, bad);
  uint64_t key[4];
  load_key(b, m, key);
  State s;
  init(s, key);
  const uint8_t* msg = b.bytes + start;
  const int64_t packets = len >> 5;
  if ((reinterpret_cast<uintptr_t>(msg) & 7) == 0) {
    const uint64_t* w = reinterpret_cast<const uint64_t*>(msg);
    for (int64_t j = 0; j < packets; ++j) {
      const uint64_t p[4] = {w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]};
      update(s, p);
    }
  } else {
    for (int64_t j = 0; j < packets; ++j) {
      uint32_t w[8];
      load_packet_bytes(msg + 32 * j, w);
      update_words(s, w);
    }
  }
  const uint32_t r = static_cast<uint32_t>(len & 31);
  uint32_t tail[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const uint8_t* t = msg + 32 * packets;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (static_cast<uint32_t>(k) < r) tail[k >> 2] |= static_cast<uint32_t>(t[k]) << (8 * (k & 3));
  }
  remainder(s, r, tail);
  finalize(s);
  store_digest(b, m, s, bad);
}

// ---------------------------------------------------------------- staged path

// Eight little-endian words of the packet at byte `off` of a staged row.
template <bool kAligned>
__device__ __forceinline__ void load_staged_packet(const uint8_t* row, uint32_t off,
                                                   uint32_t w[8]) {
  if (kAligned) {
    const uint4 a = lds128(row + off);
    const uint4 c = lds128(row + off + 16);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = c.x; w[5] = c.y; w[6] = c.z; w[7] = c.w;
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(row + (off & ~3u));
    const uint32_t sel = 0x3210u + 0x1111u * (off & 3u);
    uint32_t x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = p[i];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = __byte_perm(x[j], x[j + 1], sel);
  }
}

template <int W, int NST>
struct StagedLayout {
  static constexpr int kStride = W + 16;  // row bytes: window plus alignment slack
  static constexpr int kRowsBytes = NST * kTileRows * kStride;
  static constexpr int kPad = 64;         // packet reads may run past the last row
  static constexpr int kBytes = kRowsBytes + kPad + NST * 8;
  static_assert(kStride % 16 == 0, "rows must stay 16-byte aligned for bulk copies");
  static_assert((kStride / 4) % 32 == 4, "row stride must rotate 128-bit banks");
};

template <int W, int NST, bool kAligned>
__global__ void __launch_bounds__(kTileRows) staged_kernel(Batch b, Queue q) {
  using L = StagedLayout<W, NST>;
  constexpr int kPacketsPerStep = W / 32;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* rows = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kRowsBytes + L::kPad);
  __shared__ long long s_tile;
  __shared__ unsigned long long s_steps;

  const int t = threadIdx.x;
  resolve_count(b);
  const int64_t tiles = b.n_dev ? (b.n + kTileRows - 1) / kTileRows : q.tiles;
  if (t == 0) {
    for (int i = 0; i < NST; ++i) mbar_init(&bars[i], kTileRows);
    fence_mbar_init();
  }
  __syncthreads();

  // Whole-batch byte range: bulk copies stay inside its 16-byte aligned part;
  // the (at most two) partial 16-byte blocks at its ends are read bytewise.
  int64_t lo, hi;
  batch_range(b, lo, hi);
  const uintptr_t base = reinterpret_cast<uintptr_t>(b.bytes);
  const uintptr_t safe_lo = (base + lo + 15) & ~uintptr_t(15);
  const uintptr_t safe_hi = (base + hi) & ~uintptr_t(15);

  int issue_buf = 0;                 // buffer the next issued step goes to
  int wait_buf = 0;                  // buffer of the next step to wait for
  uint32_t wait_parity = 0;          // phase parity of that buffer
  int in_flight = 0;                 // steps issued but not yet waited for
  bool aborted = false;  // a wait ran over the limit: no more copies or hashing
  bool broken = false;   // a phase did not complete even within kDrainLimitNs
  int64_t static_tile = blockIdx.x;

  for (;;) {
    if (t == 0) {
      s_tile = q.next_tile ? static_cast<long long>(atomicAdd(q.next_tile, 1ull)) : static_tile;
      s_steps = 0;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    static_tile += gridDim.x;
    if (tile >= tiles) break;

    const int64_t idx = tile * kTileRows + t;
    const bool valid = idx < b.n;
    int64_t m = 0, start = 0, len = 0;
    int bad = 0;
    uint64_t key[4] = {0, 0, 0, 0};
    if (valid) {
      m = q.perm ? static_cast<int64_t>(q.perm[idx]) : idx;
      message_bounds(b, m, start, len, bad);
      if (bad) record_error(b.err, bad);
      load_key(b, m, key);
    }
    const int64_t my_steps = (len + W - 1) / W;
    atomicMax(&s_steps, static_cast<unsigned long long>(my_steps));
    State s;
    init(s, key);
    __syncthreads();
    const int64_t steps = static_cast<int64_t>(s_steps);

    const uintptr_t msg = base + start;
    const uint32_t mis = kAligned ? 0u : static_cast<uint32_t>(msg & 15);
    const int64_t packets = len >> 5;
    const uint32_t r = static_cast<uint32_t>(len & 31);
    const int64_t rem_step = r ? (packets * 32) / W : -1;

    // Issue step k (this thread's window [kW, min(kW + W, len)) of its message).
    auto issue = [&](int64_t k) {
      uint64_t* bar = &bars[issue_buf];
      uint8_t* row = rows + (issue_buf * kTileRows + t) * L::kStride;
      issue_buf = (issue_buf + 1 == NST) ? 0 : issue_buf + 1;
      ++in_flight;
      if (aborted || k >= my_steps) {
        mbar_arrive(bar);
        return;
      }
      const uintptr_t gs = msg + static_cast<uintptr_t>(k) * W;
      const uintptr_t ge = msg + static_cast<uintptr_t>(min(static_cast<int64_t>(k) * W + W, len));
      const uintptr_t a0 = gs & ~uintptr_t(15);
      const uintptr_t a1 = (ge + 15) & ~uintptr_t(15);
      const uintptr_t c0 = a0 > safe_lo ? a0 : safe_lo;
      const uintptr_t c1 = a1 < safe_hi ? a1 : safe_hi;
      if (c1 > c0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(c1 - c0));
        bulk_copy_g2s(row + (c0 - a0), reinterpret_cast<const void*>(c0),
                      static_cast<uint32_t>(c1 - c0), bar);
        for (uintptr_t p = gs; p < ge && p < c0; ++p)
          row[p - a0] = *reinterpret_cast<const uint8_t*>(p);
        for (uintptr_t p = (gs > c1 ? gs : c1); p < ge; ++p)
          row[p - a0] = *reinterpret_cast<const uint8_t*>(p);
      } else {
        for (uintptr_t p = gs; p < ge; ++p) row[p - a0] = *reinterpret_cast<const uint8_t*>(p);
        mbar_arrive(bar);
      }
    };

    for (int64_t k = 0; k < NST - 1 && k < steps; ++k) issue(k);
    for (int64_t k = 0; k < steps; ++k) {
      if (k + NST - 1 < steps) issue(k + NST - 1);
      const int buf = wait_buf;
      if (!broken && !mbar_wait_bounded(&bars[buf], wait_parity, b.wait_ns)) {
        // Over the limit: record the timeout, stop copying and hashing, but
        // keep waiting for this phase (bounded) so that every thread still
        // arrives exactly once per phase and no phase completes early.
        if (!aborted) record_error(b.err, kErrTimeout);
        aborted = true;
        if (!mbar_wait_bounded(&bars[buf], wait_parity, kDrainLimitNs)) broken = true;
      }
      wait_buf = (wait_buf + 1 == NST) ? 0 : wait_buf + 1;
      if (wait_buf == 0) wait_parity ^= 1u;
      --in_flight;
      if (aborted || k >= my_steps) continue;
      const uint8_t* row = rows + (buf * kTileRows + t) * L::kStride;
      const int64_t p0 = k * kPacketsPerStep;
#pragma unroll
      for (int j = 0; j < kPacketsPerStep; ++j) {
        if (p0 + j < packets) {
          uint32_t w[8];
          load_staged_packet<kAligned>(row, mis + 32u * j, w);
          update_words(s, w);
        }
      }
      if (k == rem_step) {
        uint32_t w[8];
        load_staged_packet<false>(row, mis + static_cast<uint32_t>(packets * 32 - k * W), w);
        remainder(s, r, w);
      }
    }
    finalize(s);
    if (valid) store_digest(b, m, s, bad || aborted);
    __syncthreads();  // s_tile and s_steps are rewritten for the next tile
  }

  // Phases issued but not yet waited for (only after a timeout) complete
  // before the CTA's shared memory is released.  Only a copy that never
  // lands (`broken`) can leave this loop early.
  while (in_flight > 0 && !broken) {
    mbar_wait_bounded(&bars[wait_buf], wait_parity, kDrainLimitNs);
    wait_buf = (wait_buf + 1 == NST) ? 0 : wait_buf + 1;
    if (wait_buf == 0) wait_parity ^= 1u;
    --in_flight;
  }
}

template <int W, int NST, bool kAligned>
cudaError_t launch_staged_t(const Batch& b, const Queue& q, int num_sms, cudaStream_t stream) {
  using L = StagedLayout<W, NST>;
  auto kern = staged_kernel<W, NST, kAligned>;
  cudaError_t e;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), kTileRows, L::kBytes, &e);
  if (e != cudaSuccess) return e;
  const int64_t cap = static_cast<int64_t>(per_sm) * num_sms;
  const int grid = static_cast<int>(q.tiles < cap ? q.tiles : cap);
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, kTileRows, L::kBytes, stream>>>(b, q);
  return cudaGetLastError();
}

template <int W, int NST>
int blocks_per_sm_t(bool aligned) {
  using L = StagedLayout<W, NST>;
  cudaError_t e;
  const void* kern = aligned ? reinterpret_cast<const void*>(staged_kernel<W, NST, true>)
                             : reinterpret_cast<const void*>(staged_kernel<W, NST, false>);
  return blocks_per_sm(kern, kTileRows, L::kBytes, &e);
}

}  // namespace

cudaError_t launch_naive(const Batch& b, cudaStream_t stream) {
  if (b.n <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (b.n + threads - 1) / threads;
  naive_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(b);
  return cudaGetLastError();
}

#define HH_STAGED_SHAPES(X) X(128, 3) X(128, 4) X(256, 2) X(256, 3)

cudaError_t launch_staged(const Batch& b, const Queue& q, StagedShape shape, bool aligned16,
                          int num_sms, cudaStream_t stream) {
#define HH_DISPATCH(W_, N_)                                                       \
  if (shape.window == W_ && shape.stages == N_)                                   \
    return aligned16 ? launch_staged_t<W_, N_, true>(b, q, num_sms, stream)       \
                     : launch_staged_t<W_, N_, false>(b, q, num_sms, stream);
  HH_STAGED_SHAPES(HH_DISPATCH)
#undef HH_DISPATCH
  return cudaErrorInvalidValue;
}

int staged_blocks_per_sm(StagedShape shape, bool aligned16) {
#define HH_OCC(W_, N_) \
  if (shape.window == W_ && shape.stages == N_) return blocks_per_sm_t<W_, N_>(aligned16);
  HH_STAGED_SHAPES(HH_OCC)
#undef HH_OCC
  return 0;
}

size_t staged_smem_bytes(StagedShape shape) {
#define HH_SMEM(W_, N_) \
  if (shape.window == W_ && shape.stages == N_) return StagedLayout<W_, N_>::kBytes;
  HH_STAGED_SHAPES(HH_SMEM)
#undef HH_SMEM
  return 0;
}

}  // namespace hh
