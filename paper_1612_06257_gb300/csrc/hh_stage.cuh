// hh_stage.cuh -- warp-tile staging of ragged batches, shared by the
// HighwayHash and SipTreeHash warp-tile kernels.
//
// A warp owns a tile of 32 messages (one per lane) and a private ring of NST
// shared-memory stages.  Stage k holds, per message, the 16-byte aligned
// span around bytes [kW, kW + W) of it, in the row its lane owns (W + 16
// bytes: the window plus alignment slack).  Four lanes copy each row with
// 16-byte cp.async.cg, so one instruction moves 64 contiguous bytes of each
// of 8 rows; a row's base address and chunk range come from its owner lane
// by shuffle.  Only the (at most two) partial 16-byte blocks at the two ends
// of the whole batch are read bytewise, so no load leaves [lo, hi).  When
// every row's window lies inside its message and its aligned span inside
// the batch (all but the last window of long messages), the rows copy all
// their chunks with no per-chunk tests.
#pragma once

#include <cstdint>

#include "hh_ptx.cuh"

namespace hh {

constexpr unsigned kFull = 0xffffffffu;

template <int W, int NST>
struct RaggedLayout {
  static constexpr int kStride = W + 16;             // bytes per row
  static constexpr int kChunks = kStride / 16;       // 16-byte chunks per row
  static constexpr int kPerLane = (kChunks + 3) / 4; // chunks per lane per row
  static constexpr int kStageBytes = 32 * kStride;
  static constexpr int kWarpBytes = NST * kStageBytes + 64;  // + read-past pad
  static_assert((kStride / 4) % 32 == 4, "row stride must rotate 128-bit banks");
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ int64_t warp_max(int64_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const int64_t o = __shfl_xor_sync(kFull, v, d);
    v = o > v ? o : v;
  }
  return v;
}

// The 32 bytes at byte `off` of a staged row as eight little-endian words:
// two 128-bit loads when the row is 16-byte aligned, else the nine enclosing
// 32-bit words and one PRMT per word.
template <bool kAligned>
__device__ __forceinline__ void read_packet(const uint8_t* row, uint32_t off, uint32_t w[8]) {
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

// The 17 aligned 32-bit words that hold a message of at most 64 bytes
// starting at `msg`, read straight from global memory (words past the
// message are don't-cares; shift them into place with PRMT by msg & 3).
// [lo_b, hi_b) is the batch's byte range: words that cross its ends are read
// bytewise so that no load leaves it.
__device__ __forceinline__ void load_short_words(uint32_t x[17], uintptr_t msg, uint32_t len,
                                                 uintptr_t lo_b, uintptr_t hi_b) {
  const uintptr_t w0 = msg & ~uintptr_t(3);
  const uint32_t b = static_cast<uint32_t>(msg & 3);
  const uint32_t nwords = (b + len + 3) >> 2;  // <= 17
  const uintptr_t lo4 = (lo_b + 3) & ~uintptr_t(3), hi4 = hi_b & ~uintptr_t(3);
  if (w0 >= lo4 && w0 + 68 <= hi4) {
    // All 17 words lie inside the batch: load them without per-word tests.
#pragma unroll
    for (int i = 0; i < 17; ++i) x[i] = __ldg(reinterpret_cast<const uint32_t*>(w0) + i);
  } else if (w0 >= lo4 && w0 + 4 * nwords <= hi4) {
#pragma unroll
    for (int i = 0; i < 17; ++i)
      x[i] = static_cast<uint32_t>(i) < nwords ? __ldg(reinterpret_cast<const uint32_t*>(w0) + i) : 0u;
  } else {
#pragma unroll
    for (int i = 0; i < 17; ++i) {
      uint32_t v = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uintptr_t p = w0 + 4 * i + k;
        if (static_cast<uint32_t>(i) < nwords && p >= lo_b && p < hi_b)
          v |= static_cast<uint32_t>(*reinterpret_cast<const uint8_t*>(p)) << (8 * k);
      }
      x[i] = v;
    }
  }
}

// This lane's row in each stage.  Rows rotate the banks by 4 words, so rows
// q, q + 8, q + 16, q + 24 share four banks, and two of them conflict on an
// unaligned 32-bit load when their messages start at the same word of a
// 16-byte block.  Ranking the lanes by that word (mis / 4) and giving rank q
// row q spreads equal words over the eight groups.
__device__ __forceinline__ int spread_row(bool tile_aligned, bool valid, uint32_t mis, int lane) {
  if (tile_aligned) return lane;
  const uint32_t word = valid ? (mis >> 2) : 0u;
  const unsigned below = (1u << lane) - 1u;
  int rank = 0;
#pragma unroll
  for (uint32_t v = 0; v < 4; ++v) {
    const unsigned same = __ballot_sync(kFull, word == v);
    if (v < word) rank += __popc(same);
    if (v == word) rank += __popc(same & below);
  }
  return rank;
}

// Copies the windows of a warp tile into the warp's ring (see the header).
template <int W, int NST>
struct WarpStager {
  using L = RaggedLayout<W, NST>;
  uint8_t* ring;       // the warp's ring (generic address)
  uint32_t ring_s;     // ... and its shared address
  uintptr_t msg;       // this lane's message start
  int64_t len;         // ... its length
  int64_t my_steps;    // windows it has
  int my_row;          // its row in every stage
  uintptr_t safe_lo;   // 16-byte aligned part of the batch's byte range
  uintptr_t safe_hi;
  int lane;

  // Stage k of all 32 messages into ring buffer `buf`, as one cp.async group.
  __device__ __forceinline__ void issue(int64_t k, int buf) const {
    const int part = lane & 3, row_in_pass = lane >> 2;
    // When every row's window lies inside its message and the row's whole
    // 16-byte aligned span inside the batch, all rows copy every chunk
    // (bytes past a window land in the row's slack and are never hashed).
    const uintptr_t a0_full = (msg + static_cast<uintptr_t>(k) * W) & ~uintptr_t(15);
    const bool row_full = k < my_steps && (k + 1) * W <= len && a0_full >= safe_lo &&
                          a0_full + L::kStride <= safe_hi;
    if (__all_sync(kFull, row_full)) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int owner = 8 * h + row_in_pass;
        const uintptr_t rbase = static_cast<uintptr_t>(
            __shfl_sync(kFull, static_cast<unsigned long long>(a0_full), owner));
        const int row = __shfl_sync(kFull, my_row, owner);
        const char* src = reinterpret_cast<const char*>(rbase) + 16 * part;
        const uint32_t dst = ring_s + buf * L::kStageBytes + row * L::kStride + 16 * part;
#pragma unroll
        for (int i = 0; i < L::kPerLane; ++i)
          if (i + 1 < L::kPerLane || part + 4 * i < L::kChunks)
            cp_async16(dst + 64 * i, src + 64 * i);
      }
      cp_async_commit();
      return;
    }
    uint8_t* stage = ring + buf * L::kStageBytes;
    // Owner side: this lane's window, as a 16-byte aligned chunk range.
    uintptr_t a0 = 0;
    uint32_t range = 0;  // first valid chunk | (end chunk << 8)
    if (k < my_steps) {
      const uintptr_t gs = msg + static_cast<uintptr_t>(k) * W;
      const int64_t wend = k * W + W < len ? k * W + W : len;
      const uintptr_t ge = msg + static_cast<uintptr_t>(wend);
      a0 = gs & ~uintptr_t(15);
      const uintptr_t a1 = (ge + 15) & ~uintptr_t(15);
      const uintptr_t c0 = a0 > safe_lo ? a0 : safe_lo;
      const uintptr_t c1 = a1 < safe_hi ? a1 : safe_hi;
      uint32_t first = 0, end = 0;
      if (c1 > c0) {
        first = static_cast<uint32_t>((c0 - a0) >> 4);
        end = static_cast<uint32_t>((c1 - a0) >> 4);
      }
      range = first | (end << 8);
      if (c0 > gs || c1 < ge || c1 <= c0) {
        // Bytes in the partial blocks at the batch ends: read bytewise.
        uint8_t* row = stage + my_row * L::kStride;
        for (uintptr_t p = gs; p < ge; ++p)
          if (p < c0 || p >= c1 || c1 <= c0) row[p - a0] = *reinterpret_cast<const uint8_t*>(p);
      }
    }
    // Copier side: four lanes per message, eight messages per pass.
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int owner = 8 * h + row_in_pass;
      const uintptr_t rbase = static_cast<uintptr_t>(
          __shfl_sync(kFull, static_cast<unsigned long long>(a0), owner));
      const uint32_t rr = __shfl_sync(kFull, range, owner);
      const int row = __shfl_sync(kFull, my_row, owner);
      const uint32_t first = rr & 0xff, end = rr >> 8;
      const char* src = reinterpret_cast<const char*>(rbase) + 16 * part;
      const uint32_t dst = ring_s + buf * L::kStageBytes + row * L::kStride + 16 * part;
#pragma unroll
      for (int i = 0; i < L::kPerLane; ++i) {
        const uint32_t c = part + 4 * i;
        if (c >= first && c < end) cp_async16(dst + 64 * i, src + 64 * i);
      }
    }
    cp_async_commit();
  }

  // Runs the ring over `steps` windows (the warp's longest message): stage
  // k + NST - 1 is copied while stage k is hashed by step(k, row), which
  // every lane calls for every k (its own row in stage k).
  template <typename Step>
  __device__ __forceinline__ void run(int64_t steps, Step&& step) const {
    int buf_issue = 0, buf_read = 0;
    for (int64_t k = 0; k < NST - 1; ++k) {
      if (k < steps) issue(k, buf_issue);
      else cp_async_commit();
      buf_issue = (buf_issue + 1 == NST) ? 0 : buf_issue + 1;
    }
    for (int64_t k = 0; k < steps; ++k) {
      if (k + NST - 1 < steps) issue(k + NST - 1, buf_issue);
      else cp_async_commit();
      buf_issue = (buf_issue + 1 == NST) ? 0 : buf_issue + 1;
      cp_async_wait<NST - 1>();
      __syncwarp();
      step(k, ring + buf_read * L::kStageBytes + my_row * L::kStride);
      __syncwarp();  // every lane is done with this buffer before it refills
      buf_read = (buf_read + 1 == NST) ? 0 : buf_read + 1;
    }
    cp_async_wait<0>();
  }
};

}  // namespace hh
