// hh_ragged.cu -- ragged batches: warp tiles, coalesced cp.async staging.
//
// Each warp owns a tile of 32 messages (one per lane; the 1024-bit state in
// registers) and its own ring of NST shared-memory stages, each holding a
// W-byte window of every message plus 16 bytes of alignment slack per row.
// Warps never wait on one another: no CTA barrier, a warp-private ring, and
// warp tiles taken from a queue (longest first after the length sort).
//
// Loading a stage (WarpStager, hh_stage.cuh): a message's window is the
// 16-byte aligned span around bytes [kW, kW + W) of it, in the row its lane
// owns; four lanes copy each row with 16-byte cp.async.cg, and only the
// partial 16-byte blocks at the two ends of the whole batch are read
// bytewise, so no load leaves [offsets[0], offsets[n]).
//
// Reading a packet: when every message of the warp tile starts 16-byte
// aligned, two 128-bit shared loads; otherwise the nine enclosing 32-bit
// words (eight new ones per packet: consecutive packets share one) and one
// PRMT per word to shift the bytes into place.  Rows are assigned so that
// lanes whose messages start at the same word of a 16-byte block spread over
// the shared-memory banks.
//
// Batches of messages of at most 64 bytes run in short_kernel instead (one
// thread per message, pipelined through shared memory); for large one-key
// batches short_count_kernel, which also counts the length sort's buckets.
#include <cuda_runtime.h>

#include <cstdint>

#include "hh_batch.cuh"
#include "hh_count.h"
#include "hh_device.cuh"
#include "hh_internal.h"
#include "hh_ptx.cuh"
#include "hh_stage.cuh"
#include "hh_stream.cuh"

namespace hh {
namespace {

// Hash the packets of step k that this lane's message has, from its row.
template <int W, bool kAligned>
__device__ __forceinline__ void hash_step(State& s, const uint8_t* row, uint32_t mis, int64_t k,
                                          int64_t packets, uint32_t r, int64_t rem_step,
                                          uint32_t one) {
  const int64_t p0 = k * (W / 32);
  if (kAligned) {
#pragma unroll
    for (int j = 0; j < W / 32; ++j) {
      if (p0 + j < packets) {
        uint32_t w[8];
        read_packet<true>(row, 32u * j, w);
        update_words_v<kFastUpdate>(s, w, one);
      }
    }
  } else {
    // Consecutive packets share the word that straddles them.
    const uint32_t* p = reinterpret_cast<const uint32_t*>(row + (mis & ~3u));
    const uint32_t sel = 0x3210u + 0x1111u * (mis & 3u);
    uint32_t prev = p[0];
#pragma unroll
    for (int j = 0; j < W / 32; ++j) {
      if (p0 + j < packets) {
        uint32_t x[8], w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = p[8 * j + 1 + i];
        w[0] = __byte_perm(prev, x[0], sel);
#pragma unroll
        for (int i = 1; i < 8; ++i) w[i] = __byte_perm(x[i - 1], x[i], sel);
        prev = x[7];
        update_words_v<kFastUpdate>(s, w, one);
      }
    }
  }
  if (k == rem_step) {
    uint32_t w[8];
    read_packet<false>(row, mis + static_cast<uint32_t>(packets * 32 - k * W), w);
    remainder(s, r, w);
  }
}

// Messages of at most 64 bytes (a whole warp of them), read straight from
// global memory (load_short_words): at most 17 aligned 32-bit words per
// message, shifted into place with one PRMT per word.  A message has at most
// two data Updates: a whole first packet when len > 32, then its last packet
// (padded when len mod 32 != 0).  So a warp runs at most two, whatever its
// length mix, and the padded packet is built once per message.
// hash_short_words hashes the words (b = msg & 3); hash_short loads and
// hashes.

// The last packet of a message from the eight words t that hold its last
// len mod 32 (= r) bytes, padded as Section 4.5 asks: whole 4-byte groups
// stay in place, the final r mod 4 bytes go to bytes 28.., the rest is zero.
// r == 0 leaves the whole packet t.
__device__ __forceinline__ void last_packet(uint32_t r, const uint32_t t[8], uint32_t pkt[8]) {
  const uint32_t whole = r ? (r >> 2) : 8u;
  // t[whole] for whole < 8, as a three-level select (no run-time index).
  const uint32_t w01 = (whole & 1u) ? t[1] : t[0], w23 = (whole & 1u) ? t[3] : t[2];
  const uint32_t w45 = (whole & 1u) ? t[5] : t[4], w67 = (whole & 1u) ? t[7] : t[6];
  const uint32_t w03 = (whole & 2u) ? w23 : w01, w47 = (whole & 2u) ? w67 : w45;
  const uint32_t last = (whole & 4u) ? w47 : w03;
  const uint32_t keep_last = (1u << (8u * (r & 3u))) - 1u;  // 0 when r mod 4 == 0
#pragma unroll
  for (int j = 0; j < 8; ++j) pkt[j] = (static_cast<uint32_t>(j) < whole) ? t[j] : 0u;
  pkt[7] |= last & keep_last;
}

__device__ __forceinline__ void hash_short_words(State& s, const uint32_t x[17], uint32_t b,
                                                 uint32_t len) {
  const uint32_t sel = 0x3210u + 0x1111u * b;
  uint32_t sw[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) sw[j] = __byte_perm(x[j], x[j + 1], sel);
  const bool two = len > 32u;  // a whole packet precedes the last one
  const uint32_t r = len & 31u;
  uint32_t t[8], last[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) t[j] = two ? sw[8 + j] : sw[j];
  last_packet(r, t, last);
  if (two) {
    const uint32_t* first = sw;
    update_words(s, first);
  }
  if (len != 0u) {
    inject_size(s, r);  // a size of 0 changes nothing
    update_words(s, last);
  }
}

// As hash_short_words, reading the 17 staged words from a shared-memory slot:
// the last packet's nine words are read from word 8 when a whole packet
// precedes it (no select between the two windows), and the word that holds
// the final len mod 4 bytes is read at its own index (no select tree).
__device__ __forceinline__ void hash_short_slot(State& s, const uint32_t* slot, uint32_t b,
                                                uint32_t len) {
  const uint32_t sel = 0x3210u + 0x1111u * b;
  const bool two = len > 32u;
  const uint32_t r = len & 31u;
  const uint32_t* lp = slot + (two ? 8 : 0);
  uint32_t t[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) t[j] = __byte_perm(lp[j], lp[j + 1], sel);
  const uint32_t whole = r ? (r >> 2) : 8u;
  const uint32_t wl = whole < 7u ? whole : 7u;
  const uint32_t last = __byte_perm(lp[wl], lp[wl + 1], sel);
  const uint32_t keep_last = (1u << (8u * (r & 3u))) - 1u;  // 0 when r mod 4 == 0
  uint32_t pkt[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) pkt[j] = (static_cast<uint32_t>(j) < whole) ? t[j] : 0u;
  pkt[7] |= last & keep_last;
  if (two) {
    uint32_t f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = __byte_perm(slot[j], slot[j + 1], sel);
    update_words(s, f);
  }
  if (len != 0u) {
    inject_size(s, r);
    update_words(s, pkt);
  }
}

__device__ __forceinline__ void hash_short(State& s, uintptr_t msg, uint32_t len, uintptr_t lo_b,
                                           uintptr_t hi_b) {
  uint32_t x[17];
  load_short_words(x, msg, len, lo_b, hi_b);
  hash_short_words(s, x, static_cast<uint32_t>(msg & 3), len);
}

// Starts copying the 17 words that hold a message of at most 64 bytes into
// a thread's shared-memory slot (slot_s is its shared address), as one
// cp.async group; words that cross the batch ends are read now, bytewise.
__device__ __forceinline__ void stage_short_words(uint32_t* slot, uint32_t slot_s, uintptr_t msg,
                                                  uint32_t len, uintptr_t lo_b, uintptr_t hi_b) {
  const uintptr_t w0 = msg & ~uintptr_t(3);
  const uintptr_t lo4 = (lo_b + 3) & ~uintptr_t(3), hi4 = hi_b & ~uintptr_t(3);
  if (w0 >= lo4 && w0 + 68 <= hi4) {
#pragma unroll
    for (int i = 0; i < 17; ++i) cp_async4(slot_s + 4 * i, reinterpret_cast<const uint32_t*>(w0) + i);
  } else {
    uint32_t x[17];
    load_short_words(x, msg, len, lo_b, hi_b);
#pragma unroll
    for (int i = 0; i < 17; ++i) slot[i] = x[i];
  }
  cp_async_commit();
}

// Half of a 32-byte packet: the 16 bytes at byte `off` of a row, as two
// little-endian 64-bit lanes.
template <bool kAligned>
__device__ __forceinline__ void read_half_packet(const uint8_t* row, uint32_t off, uint64_t& p0,
                                                 uint64_t& p1) {
  if (kAligned) {
    const uint4 a = lds128(row + off);
    p0 = join(a.x, a.y);
    p1 = join(a.z, a.w);
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(row + (off & ~3u));
    const uint32_t sel = 0x3210u + 0x1111u * (off & 3u);
    uint32_t x[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) x[i] = p[i];
    p0 = join(__byte_perm(x[0], x[1], sel), __byte_perm(x[1], x[2], sel));
    p1 = join(__byte_perm(x[2], x[3], sel), __byte_perm(x[3], x[4], sel));
  }
}

// One pair tile: messages [first, last) (at most 16) of the huge prefix of
// the length order, two lanes per message (lane 2s + h keeps lanes 2h, 2h+1
// of message first + s's state).
// Each message's row spans two ring rows and holds a 2W-byte window.
template <int W, int NST>
__device__ __forceinline__ void pair_tile(const Batch& b, const int32_t* perm, int64_t first,
                                          int64_t last, uint8_t* ring, uint32_t ring_s,
                                          uintptr_t base, uintptr_t safe_lo, uintptr_t safe_hi,
                                          int lane) {
  using L = RaggedLayout<W, NST>;
  constexpr int WP = 2 * W;                   // window bytes per step
  constexpr int kRowStride = 2 * L::kStride;  // one message row = two ring rows
  constexpr int kChunks = WP / 16 + 1;
  constexpr int kPerLane = (kChunks + 3) / 4;
  const int slot = lane >> 1, half = lane & 1;
  const int64_t idx = first + slot;
  const bool valid = idx < last;
  int64_t m = 0, start = 0, len = 0;
  int bad = 0;
  if (valid) {
    m = static_cast<int64_t>(perm[idx]);
    message_bounds(b, m, start, len, bad);
    if (bad && half == 0) record_error(b.err, bad);
  }
  Half s;
  start_half(b, m, valid, half, s);
  const int64_t my_steps = (len + WP - 1) / WP;
  const int64_t steps = warp_max(my_steps);
  const uintptr_t msg = base + start;
  const uint32_t mis = static_cast<uint32_t>(msg & 15);
  const bool aligned = __all_sync(kFull, mis == 0 || !valid);
  const int64_t packets = len >> 5;
  const uint32_t r = static_cast<uint32_t>(len & 31);
  const int64_t rem_step = r ? (packets * 32) / WP : -1;
  const int part = lane & 3, slot_in_pass = lane >> 2;

  auto issue = [&](int64_t k, int buf) {
    uint8_t* stage = ring + buf * L::kStageBytes;
    uintptr_t a0 = 0;
    uint32_t range = 0;
    if (half == 0 && k < my_steps) {
      const uintptr_t gs = msg + static_cast<uintptr_t>(k) * WP;
      const int64_t wend = k * WP + WP < len ? k * WP + WP : len;
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
        uint8_t* row = stage + slot * kRowStride;
        for (uintptr_t p = gs; p < ge; ++p)
          if (p < c0 || p >= c1 || c1 <= c0) row[p - a0] = *reinterpret_cast<const uint8_t*>(p);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = 8 * h + slot_in_pass;
      const uintptr_t rbase = static_cast<uintptr_t>(
          __shfl_sync(kFull, static_cast<unsigned long long>(a0), 2 * row));
      const uint32_t rr = __shfl_sync(kFull, range, 2 * row);
      const uint32_t first = rr & 0xff, end = rr >> 8;
      const char* src = reinterpret_cast<const char*>(rbase) + 16 * part;
      const uint32_t dst = ring_s + buf * L::kStageBytes + row * kRowStride + 16 * part;
#pragma unroll
      for (int i = 0; i < kPerLane; ++i) {
        const uint32_t c = part + 4 * i;
        if (c >= first && c < end) cp_async16(dst + 64 * i, src + 64 * i);
      }
    }
    cp_async_commit();
  };

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
    const int64_t left = packets - k * (WP / 32);
    // Every message of the tile has a full window: constant trip count.
    const bool full = __all_sync(kFull, !valid || left >= WP / 32);
    if (k < my_steps) {
      const uint8_t* row = ring + buf_read * L::kStageBytes + slot * kRowStride;
      const int count = left < WP / 32 ? static_cast<int>(left) : WP / 32;
      if (full && aligned) {
        const uint8_t* hrow = row + 16u * half;
#pragma unroll
        for (int j = 0; j < WP / 32; ++j) {
          uint64_t x0, x1;
          read_half_packet<true>(hrow, 32u * j, x0, x1);
          update_half(s, x0, x1);
        }
      } else if (full) {
        const uint32_t off = mis + 16u * half;
#pragma unroll
        for (int j = 0; j < WP / 32; ++j) {
          uint64_t x0, x1;
          read_half_packet<false>(row, off + 32u * j, x0, x1);
          update_half(s, x0, x1);
        }
      } else if (aligned) {
#pragma unroll 4
        for (int j = 0; j < count; ++j) {
          uint64_t x0, x1;
          read_half_packet<true>(row, 32u * j + 16u * half, x0, x1);
          update_half(s, x0, x1);
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < count; ++j) {
          uint64_t x0, x1;
          read_half_packet<false>(row, mis + 32u * j + 16u * half, x0, x1);
          update_half(s, x0, x1);
        }
      }
      if (k == rem_step) {
        uint32_t w[8], rp[8];
        read_packet<false>(row, mis + static_cast<uint32_t>(packets * 32 - k * WP), w);
        remainder_packet(r, w, rp);
        inject_size_half(s, r);
        if (half == 0) update_half(s, join(rp[0], rp[1]), join(rp[2], rp[3]));
        else update_half(s, join(rp[4], rp[5]), join(rp[6], rp[7]));
      }
    }
    __syncwarp();
    buf_read = (buf_read + 1 == NST) ? 0 : buf_read + 1;
  }
  cp_async_wait<0>();
  end_half(b, m, valid, bad, half, s);
  __syncwarp();
}

// One solo tile: a single message of the huge prefix owns the whole warp.
// Lanes 0 and 1 hash it (one lane pair each, as in a pair tile); all 32
// lanes copy it, and realign each stage in shared memory when the message
// does not start on a 16-byte boundary.  The warp's ring is re-cut into kSoloStages stages of 8W
// bytes, so about 14 KiB (W = 256) of the message is in flight and the
// copies never hold up the Update chain, which then runs at the rate one
// warp issues it.  Used while the huge messages are few enough to get a
// warp scheduler each (Queue::solo_max).
constexpr int kSoloStages = 8;

// Solo tiles running on this device, over every ragged kernel in flight,
// the ragged launches with huge messages in flight, and which warp
// schedulers run a solo tile (slot = 4 * SM + hardware warp slot mod 4).
__device__ unsigned int g_solo_active = 0;
__device__ unsigned int g_huge_kernels = 0;
constexpr int kSchedulerSlots = 4096;
__device__ unsigned int g_scheduler_solo[kSchedulerSlots];

// This warp's scheduler slot (a placement hint only: results never depend
// on it).
__device__ __forceinline__ unsigned scheduler_slot() {
  unsigned sm, warp;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
  asm volatile("mov.u32 %0, %%warpid;" : "=r"(warp));
  return (4u * sm + (warp & 3u)) & (kSchedulerSlots - 1);
}

template <int W, int NST>
__device__ __forceinline__ void solo_tile(const Batch& b, const int32_t* perm, int64_t tile,
                                          uint8_t* ring, uint32_t ring_s, uintptr_t base,
                                          uintptr_t safe_lo, uintptr_t safe_hi, int lane) {
  constexpr int SW = 8 * W;               // window bytes per stage
  constexpr int kRow = SW + 16;           // 16-byte aligned span of a window
  constexpr int kChunks = kRow / 16;
  constexpr int kPerLane = (kChunks + 31) / 32;
  static_assert(kSoloStages * kRow + 64 <= RaggedLayout<W, NST>::kWarpBytes,
                "solo stages (and the read-past pad) must fit the warp's ring");
  const int half = lane & 1;
  const int64_t m = static_cast<int64_t>(perm[tile]);
  int64_t start = 0, len = 0;
  int bad = 0;
  message_bounds(b, m, start, len, bad);
  if (bad && lane == 0) record_error(b.err, bad);
  Half s;
  start_half(b, m, true, half, s);
  const int64_t steps = (len + SW - 1) / SW;
  const uintptr_t msg = base + start;
  const uint32_t mis = static_cast<uint32_t>(msg & 15);
  const int64_t packets = len >> 5;
  const uint32_t r = static_cast<uint32_t>(len & 31);
  const int64_t rem_step = r ? (packets * 32) / SW : -1;

  auto issue = [&](int64_t k, int buf) {
    const uintptr_t gs = msg + static_cast<uintptr_t>(k) * SW;
    const int64_t wend = k * SW + SW < len ? k * SW + SW : len;
    const uintptr_t ge = msg + static_cast<uintptr_t>(wend);
    const uintptr_t a0 = gs & ~uintptr_t(15);
    const uintptr_t a1 = (ge + 15) & ~uintptr_t(15);
    const uintptr_t c0 = a0 > safe_lo ? a0 : safe_lo;
    const uintptr_t c1 = a1 < safe_hi ? a1 : safe_hi;
    uint32_t first = 0, end = 0;
    if (c1 > c0) {
      first = static_cast<uint32_t>((c0 - a0) >> 4);
      end = static_cast<uint32_t>((c1 - a0) >> 4);
    }
    const uint32_t dst = ring_s + buf * kRow;
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
      const uint32_t c = static_cast<uint32_t>(lane + 32 * i);
      if (c >= first && c < end)
        cp_async16(dst + 16 * c, reinterpret_cast<const char*>(a0) + 16 * c);
    }
    // The (at most two) partial 16-byte blocks at the ends of the batch.
    if (lane == 0 && (c0 > gs || c1 < ge || c1 <= c0)) {
      uint8_t* row = ring + buf * kRow;
      for (uintptr_t p = gs; p < ge; ++p)
        if (p < c0 || p >= c1 || c1 <= c0) row[p - a0] = *reinterpret_cast<const uint8_t*>(p);
    }
    cp_async_commit();
  };

  int buf_issue = 0, buf_read = 0;
  for (int64_t k = 0; k < kSoloStages - 1; ++k) {
    if (k < steps) issue(k, buf_issue);
    else cp_async_commit();
    buf_issue = (buf_issue + 1 == kSoloStages) ? 0 : buf_issue + 1;
  }
  for (int64_t k = 0; k < steps; ++k) {
    if (k + kSoloStages - 1 < steps) issue(k + kSoloStages - 1, buf_issue);
    else cp_async_commit();
    buf_issue = (buf_issue + 1 == kSoloStages) ? 0 : buf_issue + 1;
    cp_async_wait<kSoloStages - 1>();
    __syncwarp();
    uint8_t* row = ring + buf_read * kRow;
    if (mis != 0) {
      // All 32 lanes shift the stage left by `mis` bytes in place, so the
      // two hashing lanes read aligned 16-byte words.  Lane i makes output
      // words i, i + 32, ... (consecutive lanes touch consecutive words: no
      // bank conflicts), each from two input words and one PRMT; every lane
      // reads before any lane writes.  Reads stay inside the row (its 16
      // slack bytes cover the shift); bytes past the window are never hashed.
      constexpr int kPerLane = SW / 4 / 32;
      const uint32_t q = mis >> 2;
      const uint32_t sel = 0x3210u + 0x1111u * (mis & 3u);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(row) + q;
      uint32_t y[kPerLane];
#pragma unroll
      for (int j = 0; j < kPerLane; ++j)
        y[j] = __byte_perm(src[lane + 32 * j], src[lane + 32 * j + 1], sel);
      __syncwarp();
      uint32_t* dst = reinterpret_cast<uint32_t*>(row);
#pragma unroll
      for (int j = 0; j < kPerLane; ++j) dst[lane + 32 * j] = y[j];
      __syncwarp();
    }
    if (lane < 2) {
      const int64_t left = packets - k * (SW / 32);
      if (left >= SW / 32) {
        // A full stage: constant trip count, offsets fold into the loads.
        const uint8_t* hrow = row + 16u * half;
#pragma unroll 16
        for (int j = 0; j < SW / 32; ++j) {
          uint64_t x0, x1;
          read_half_packet<true>(hrow, 32u * j, x0, x1);
          update_half(s, x0, x1);
        }
      } else {
        const int count = static_cast<int>(left);
#pragma unroll 4
        for (int j = 0; j < count; ++j) {
          uint64_t x0, x1;
          read_half_packet<true>(row, 32u * j + 16u * half, x0, x1);
          update_half(s, x0, x1);
        }
      }
      if (k == rem_step) {
        uint32_t w[8], rp[8];
        read_packet<true>(row, static_cast<uint32_t>(packets * 32 - k * SW), w);
        remainder_packet(r, w, rp);
        inject_size_half(s, r);
        if (half == 0) update_half(s, join(rp[0], rp[1]), join(rp[2], rp[3]));
        else update_half(s, join(rp[4], rp[5]), join(rp[6], rp[7]));
      }
    }
    __syncwarp();
    buf_read = (buf_read + 1 == kSoloStages) ? 0 : buf_read + 1;
  }
  cp_async_wait<0>();
  end_half(b, m, lane < 2, bad, half, s);
  __syncwarp();
}

// kHuge: the variant with the huge-message phase (solo and pair tiles).
// Without it the warp-tile code needs fewer registers (144 against 167 at
// 256-byte windows) and runs faster.  For large sorted batches both variants
// are launched (q.skip_if_short set, as for the short kernel) and each
// returns at once unless the sort's count of huge messages is its case;
// otherwise only the variant with the phase is launched and does all work.
template <int W, int NST, int WARPS, bool kHuge>
__global__ void __launch_bounds__(WARPS * 32, 2) ragged_kernel(Batch b, Queue q) {
  using L = RaggedLayout<W, NST>;
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* ring = smem + warp * L::kWarpBytes;
  const uint32_t ring_s = smem_u32(ring);
  resolve_count(b);

  int64_t lo, hi;
  batch_range(b, lo, hi);
  const uintptr_t base = reinterpret_cast<uintptr_t>(b.bytes);
  const uintptr_t safe_lo = (base + lo + 15) & ~uintptr_t(15);
  const uintptr_t safe_hi = (base + hi) & ~uintptr_t(15);

  if (q.skip_if_short && q.use_perm != nullptr && *q.use_perm == 0) return;  // short kernel runs
  const int32_t* perm = (q.perm && (q.use_perm == nullptr || *q.use_perm)) ? q.perm : nullptr;
  // The huge prefix of the length order (messages perm[0 .. huge)) comes
  // first, then warp tiles of 32 messages from counter next_tile[0].
  const int64_t huge = (perm != nullptr && q.huge_count != nullptr) ? *q.huge_count : 0;
  if (q.skip_if_short && (huge > 0) != kHuge) return;  // the other variant runs
  const int64_t tiles = (b.n - huge + 31) / 32;
  int64_t static_tile = static_cast<int64_t>(blockIdx.x) * WARPS + warp;
  const int64_t static_step = static_cast<int64_t>(gridDim.x) * WARPS;

  // Huge messages, longest first, claimed with fetch-and-add on
  // next_tile[1]: a solo tile takes one message, a pair tile 16.  Solo
  // tiles are taken only by warps of blocks 0 .. solo_ctas - 1 (the first
  // wave places those blocks one per SM), on a warp scheduler that runs no
  // other solo tile (g_scheduler_solo, over all launches in flight), while
  // fewer than q.solo_max solo tiles run on the device (g_solo_active), and, unless q.solo_shared, only while no other launch
  // with huge messages is in flight (g_huge_kernels, which a launch joins
  // through next_tile[2] and leaves when its last warp, counted in
  // next_tile[3], is done): under load, one message per warp would waste
  // the issue slots that a pair tile shares among 16 messages.  Warps of
  // other blocks skip this phase when solo tiles can take the whole prefix.
  // Warps of the solo blocks leave it only when nothing is left, so every
  // huge message is claimed.
  if (kHuge && huge > 0 && q.next_tile != nullptr) {
    const bool eligible = q.solo_max > 0 && static_cast<int>(blockIdx.x) < q.solo_ctas;
    int alone = 0;
    if (lane == 0) {
      if (atomicCAS(q.next_tile + 2, 0ull, 1ull) == 0ull) atomicAdd(&g_huge_kernels, 1u);
      // 0 can be read while this launch's own join is still in flight.
      alone = q.solo_shared || atomicAdd(&g_huge_kernels, 0u) <= 1u;
    }
    alone = __shfl_sync(kFull, alone, 0);
    const bool all_solo = alone && huge <= q.solo_max;
    const unsigned slot = scheduler_slot();
    while (eligible || !all_solo) {
      int kind = 0;  // 0: nothing left, 1: solo, 2: pair
      long long first = 0, last = 0;
      if (lane == 0) {
        bool solo = false;
        if (eligible && (q.solo_shared || atomicAdd(&g_huge_kernels, 0u) <= 1u)) {
          // A solo tile needs a scheduler with no other solo tile on it.
          solo = atomicCAS(&g_scheduler_solo[slot], 0u, 1u) == 0u;
          if (solo && atomicAdd(&g_solo_active, 1u) >= static_cast<unsigned>(q.solo_max)) {
            atomicSub(&g_solo_active, 1u);
            atomicExch(&g_scheduler_solo[slot], 0u);
            solo = false;
          }
        }
        const unsigned long long take = solo ? 1ull : 16ull;
        const long long f = static_cast<long long>(atomicAdd(q.next_tile + 1, take));
        if (f < huge) {
          kind = solo ? 1 : 2;
          first = f;
          last = f + static_cast<long long>(take) < huge ? f + static_cast<long long>(take) : huge;
        } else if (solo) {
          atomicSub(&g_solo_active, 1u);
          atomicExch(&g_scheduler_solo[slot], 0u);
        }
      }
      kind = __shfl_sync(kFull, kind, 0);
      if (kind == 0) break;
      first = __shfl_sync(kFull, first, 0);
      last = __shfl_sync(kFull, last, 0);
      if (kind == 1) {
        solo_tile<W, NST>(b, perm, first, ring, ring_s, base, safe_lo, safe_hi, lane);
        if (lane == 0) {
          atomicSub(&g_solo_active, 1u);
          atomicExch(&g_scheduler_solo[slot], 0u);
        }
      } else {
        pair_tile<W, NST>(b, perm, first, last, ring, ring_s, base, safe_lo, safe_hi, lane);
      }
    }
  }

  for (;;) {
    int64_t tile;
    if (q.next_tile) {
      unsigned long long tk = 0;
      if (lane == 0) tk = atomicAdd(q.next_tile, 1ull);
      tile = static_cast<int64_t>(__shfl_sync(kFull, tk, 0));
    } else {
      tile = static_tile;
      static_tile += static_step;
    }
    if (tile >= tiles) break;

    const int64_t idx = huge + tile * 32 + lane;
    const bool valid = idx < b.n;
    int64_t m = 0, start = 0, len = 0;
    int bad = 0;
    if (valid) {
      m = perm ? static_cast<int64_t>(perm[idx]) : idx;
      message_bounds(b, m, start, len, bad);
      if (bad) record_error(b.err, bad);
    }
    State s;
    start_state(b, m, valid, s);
    if (__all_sync(kFull, len <= 64)) {
      hash_short(s, base + start, static_cast<uint32_t>(len), base + lo, base + hi);
      end_state(b, m, valid, bad, s);
      continue;
    }
    const int64_t my_steps = (len + W - 1) / W;
    const int64_t steps = warp_max(my_steps);
    const uintptr_t msg = base + start;
    const uint32_t mis = static_cast<uint32_t>(msg & 15);
    const bool aligned = __all_sync(kFull, mis == 0 || !valid);
    const int64_t packets = len >> 5;
    const uint32_t r = static_cast<uint32_t>(len & 31);
    const int64_t rem_step = r ? (packets * 32) / W : -1;
    const WarpStager<W, NST> stager{ring, ring_s, msg, len, my_steps,
                                    spread_row(aligned, valid, mis, lane), safe_lo, safe_hi,
                                    lane};
    stager.run(steps, [&](int64_t k, const uint8_t* row) {
      if (k < my_steps) {
        if (aligned)  // warp-uniform
          hash_step<W, true>(s, row, 0u, k, packets, r, rem_step, 1u);
        else
          hash_step<W, false>(s, row, mis, k, packets, r, rem_step, 1u);
      }
    });
    end_state(b, m, valid, bad, s);
    __syncwarp();
  }
  // The last warp of a launch with huge messages leaves g_huge_kernels.
  if (kHuge && huge > 0 && q.next_tile != nullptr && lane == 0 &&
      atomicAdd(q.next_tile + 3, 1ull) == static_cast<unsigned long long>(gridDim.x) * WARPS - 1)
    atomicSub(&g_huge_kernels, 1u);
}

// The hash of message m from its finalised state (zero for an invalid
// descriptor): kWords output words (b.words), or b.words read at run time
// when kWords is 0.  With kWords known, only lanes 0 .. kWords - 1 of the
// final state are live, and the compiler drops the finalisation work that
// feeds no stored lane: for 64- and 128-bit output, all of the last round's
// second lane pair and most of the one before.
template <int kWords>
__device__ __forceinline__ void store_short_hash(const Batch& b, int64_t m, int bad,
                                                 const State& s) {
  const uint64_t keep = bad ? 0ull : ~0ull;
  const int words = kWords ? kWords : b.words;
  uint64_t* o = b.out + m * words;
  o[0] = (s.v0[0] + s.v1[0] + s.mul0[0] + s.mul1[0]) & keep;
  if (words >= 2) o[1] = (s.v0[1] + s.v1[1] + s.mul0[1] + s.mul1[1]) & keep;
  if (words == 4) {
    o[2] = (s.v0[2] + s.v1[2] + s.mul0[2] + s.mul1[2]) & keep;
    o[3] = (s.v0[3] + s.v1[3] + s.mul0[3] + s.mul1[3]) & keep;
  }
}

// Thread per message for batches whose messages are all at most kShortMax
// bytes, other than the one-key offsets-form batches that short_count_kernel
// takes: a key per message, a key table, segments and streams.  In index
// order (neighbouring threads read neighbouring bytes), three blocks of 256
// threads per SM (80 registers).  kWords: the output width in words, fixed
// per instantiation for whole messages (0 in the stream instantiation, which
// reads it at run time).
template <bool kStream, int kWords>
__global__ void __launch_bounds__(256, kStream ? 2 : 3) short_kernel(Batch b, const int* run_if) {
  if (run_if != nullptr && *run_if != 0) return;
  resolve_count(b);
  int64_t lo, hi;
  batch_range(b, lo, hi);
  const uintptr_t base = reinterpret_cast<uintptr_t>(b.bytes);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t first_m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (kStream || b.offsets == nullptr || b.key_index != nullptr) {
    for (int64_t m = first_m; m < b.n; m += stride) {
      int64_t s0, len;
      int bad;
      message_bounds(b, m, s0, len, bad);
      if (bad) record_error(b.err, bad);
      len = len < kShortMax ? len : kShortMax;
      State s;
      start_state(b, m, true, s);
      hash_short(s, base + s0, static_cast<uint32_t>(len), base + lo, base + hi);
      end_state(b, m, true, bad, s);
    }
    return;
  }
  // Offsets form, pipelined one message ahead: at the start of a message the
  // thread copies the next message's two offsets into shared memory, so that
  // no message waits for its offsets.  The words are loaded directly: the
  // key load is waited for anyway, and staging the words measured slower.
  __shared__ int64_t next_offsets[2][256][2];
  const int tid = threadIdx.x;
  auto fetch_offsets = [&](int64_t mm, int slot) {
    cp_async8(smem_u32(&next_offsets[slot][tid][0]), b.offsets + mm);
    cp_async8(smem_u32(&next_offsets[slot][tid][1]), b.offsets + mm + 1);
    cp_async_commit();
  };
  if (first_m < b.n) fetch_offsets(first_m, 0);
  int cur = 0;
  for (int64_t m = first_m; m < b.n; m += stride) {
    cp_async_wait<0>();
    const int64_t s0 = next_offsets[cur][tid][0], e0 = next_offsets[cur][tid][1];
    if (m + stride < b.n) fetch_offsets(m + stride, cur ^ 1);
    cur ^= 1;
    const int bad = e0 < s0 ? kErrBadOffsets : 0;
    int64_t len = bad ? 0 : e0 - s0;
    len = len < kShortMax ? len : kShortMax;
    if (bad) record_error(b.err, bad);
    const uint64_t* kp = key_of(b, m);
    uint64_t key[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = __ldg(kp + i);
    State s;
    init(s, key);
    hash_short(s, base + s0, static_cast<uint32_t>(len), base + lo, base + hi);
    finalize(s);
    store_short_hash<kWords>(b, m, bad, s);
  }
}

// The flag that some message is longer than kShortMax: relaxed GPU-scope
// accesses, so that a store on one SM reaches the loads of the others.
__device__ __forceinline__ uint32_t load_flag(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void set_flag(uint32_t* p) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(1u) : "memory");
}

// short_kernel's one-key offsets-form loop with the length count of the
// sort folded in (one pass over the offsets instead of two).
//
// Work: runs of kRunMsgs consecutive messages, kRun per lane (lane l takes
// messages base + 32 j + l, so a warp's loads and stores stay coalesced).
// A warp's two first runs follow from its index (run k of warp w is number
// k W + w, W warps in the grid); the later ones come from a counter
// (hist[kBuckets + 1]), each claimed a run ahead (a claim for the first run,
// made by every warp at kernel start on one word, took 10 us of a
// 2^20-message count).  With a fixed share per thread the warps that the
// scheduler favoured finished early and left the SMs short of warps (17.8
// of 24 active on average).
//
// Count: buckets 0..2 (messages of at most kShortMax bytes, whose order
// among themselves does not matter) are merged into bucket 2, as the
// scatter of this path does; a longer message goes to its own bucket
// (bucket_of_packets of ceil(len / 32)).
//
// Hash: a message of at most kShortMax bytes is hashed (and tallied for
// bucket 2) until a lane of the warp meets a longer one, which sets the flag
// hist[kBuckets] (one store per block), or the warp finds the flag set (read
// once per run, a run ahead, from a warp's third run on).  From then on the
// warp only counts, four messages per lane per step with their offsets
// loaded together.  A set flag means a long message is in the histogram:
// the scan turns the sorted order on and the warp-tile kernel hashes every
// message, so none skipped here goes unhashed.  In an all-short batch
// nothing sets the flag and every message is hashed here.  The block's
// histogram reuses the staged-word buffer once the block's threads are done
// hashing (each with its copies landed), so the kernel takes no more shared
// memory, and L1 no less, than short_kernel.
constexpr uint32_t kRun = 8;
constexpr uint32_t kRunMsgs = 32 * kRun;
constexpr uint32_t kCountWarps = 8;  // warps per block

template <int kWords>
__global__ void __launch_bounds__(256, 3) short_count_kernel(Batch b, uint32_t* hist) {
  // Message indices fit in 32 bits: a sorted batch has at most 2^31 - 1
  // messages, and the runs handed out pass n by at most two per warp.
  const uint32_t n = static_cast<uint32_t>(b.n);
  int64_t lo, hi;
  batch_range(b, lo, hi);
  const uintptr_t base = reinterpret_cast<uintptr_t>(b.bytes);
  uint32_t* flag = hist + kBuckets;
  uint32_t* run_counter = hist + kBuckets + 1;
  __shared__ int64_t next_offsets[2][256][2];
  __shared__ uint32_t next_words[2][256 * 17];
  __shared__ __align__(16) uint64_t s_init[16];
  __shared__ uint32_t s_told;  // the block has stored the flag
  static_assert(sizeof(next_words) >= kBuckets * sizeof(uint32_t), "histogram space");
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  if (tid == 0) {
    s_told = 0;
    uint64_t key[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = __ldg(b.keys + i);
    State s0;
    init(s0, key);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s_init[i] = s0.v0[i];
      s_init[4 + i] = s0.v1[i];
      s_init[8 + i] = s0.mul0[i];
      s_init[12 + i] = s0.mul1[i];
    }
  }
  __syncthreads();
  auto fetch_offsets = [&](uint32_t mm, int slot) {
    cp_async8(smem_u32(&next_offsets[slot][tid][0]), b.offsets + mm);
    cp_async8(smem_u32(&next_offsets[slot][tid][1]), b.offsets + mm + 1);
    cp_async_commit();
  };
  auto fetch_words = [&](int slot) {  // the slot's offsets have landed
    const int64_t s = next_offsets[slot][tid][0], e = next_offsets[slot][tid][1];
    const int64_t l = e < s ? 0 : e - s;
    if (l > kShortMax) return;  // only counted
    uint32_t* dst = &next_words[slot][17 * tid];
    stage_short_words(dst, smem_u32(dst), base + s, static_cast<uint32_t>(l), base + lo, base + hi);
  };
  // A warp's two first runs go by its index (half of fixed_end apart); the
  // counter hands out the runs from fixed_end on, each claimed a run ahead
  // (ticket: lane 0's claim for the run after next_run).
  const uint32_t fixed_end = 2 * gridDim.x * kCountWarps * kRunMsgs;
  uint32_t run = (blockIdx.x * kCountWarps + (tid >> 5)) * kRunMsgs;
  uint32_t next_run = run + fixed_end / 2;
  uint32_t ticket = 0;
  if (lane == 0) ticket = atomicAdd(run_counter, kRunMsgs);
  auto advance = [&]() {
    run = next_run;
    next_run = fixed_end + __shfl_sync(0xffffffffu, ticket, 0);
    if (lane == 0) ticket = atomicAdd(run_counter, kRunMsgs);
  };
  uint32_t m = run + lane;
  uint32_t j = 0;
  uint32_t hashed = 0;  // messages hashed here (all in bucket 2)
  if (m < n) {
    fetch_offsets(m, 0);
    cp_async_wait<0>();
    fetch_words(0);
  }
  int cur = 0;
  uint32_t seen = 0;  // the flag as read during the run before
  while (run < n) {
    if (__any_sync(0xffffffffu, seen != 0)) break;  // count from step 0 of this run
    if (run >= fixed_end) seen = load_flag(flag);  // not in the warp's fixed runs
    bool met_long = false;
    for (j = 0; j < kRun; ++j, m += 32) {
      cp_async_wait<0>();  // this message's offsets and words are in slot cur
      const bool have = m < n;
      const int64_t s0 = next_offsets[cur][tid][0], e0 = next_offsets[cur][tid][1];
      const int bad = have && e0 < s0 ? kErrBadOffsets : 0;
      const int64_t len = bad || !have ? 0 : e0 - s0;
      const bool is_long = len > kShortMax;
      if (__any_sync(0xffffffffu, is_long)) {  // the warp counts from here on
        if (is_long && atomicExch(&s_told, 1u) == 0u) set_flag(flag);
        met_long = true;
        break;
      }
      const uint32_t nm = j + 1 < kRun ? m + 32 : next_run + lane;
      const bool more = nm < n;
      if (more) fetch_offsets(nm, cur ^ 1);
      if (bad) record_error(b.err, bad);
      hashed += have ? 1u : 0u;
      State s;
      {
        const uint4* p = reinterpret_cast<const uint4*>(s_init);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const uint4 a = p[i], c = p[2 + i], d = p[4 + i], e = p[6 + i];
          s.v0[2 * i] = join(a.x, a.y);
          s.v0[2 * i + 1] = join(a.z, a.w);
          s.v1[2 * i] = join(c.x, c.y);
          s.v1[2 * i + 1] = join(c.z, c.w);
          s.mul0[2 * i] = join(d.x, d.y);
          s.mul0[2 * i + 1] = join(d.z, d.w);
          s.mul1[2 * i] = join(e.x, e.y);
          s.mul1[2 * i + 1] = join(e.z, e.w);
        }
      }
      hash_short_slot(s, &next_words[cur][17 * tid], static_cast<uint32_t>((base + s0) & 3),
                      static_cast<uint32_t>(len));
      if (more) {
        cp_async_wait<0>();
        fetch_words(cur ^ 1);
      }
      cur ^= 1;
      finalize(s);
      if (have) store_short_hash<kWords>(b, m, bad, s);
    }
    if (met_long) break;  // count from step j of this run
    advance();
    m = run + lane;
    j = 0;
  }
  // Count only: this run from step j on (message m, not counted yet), then
  // the runs that follow.  Runs of equal buckets go to the block histogram
  // with one shared atomic per run; it takes the staged-word buffer once
  // every thread of the block is done with it.
  cp_async_wait<0>();
  __syncthreads();
  uint32_t* h = &next_words[0][0];
  for (int i = tid; i < kBuckets; i += 256) h[i] = 0;
  __syncthreads();
  uint32_t short_count = hashed;
  int run_key = 0;
  uint32_t same = 0;
  while (run < n) {
    for (; j < kRun; j += 4, m += 128) {
      int64_t st[4], en[4];
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t i = m + 32 * q;
        const uint32_t k = i < n ? i : n - 1;
        st[q] = __ldg(b.offsets + k);
        en[q] = __ldg(b.offsets + k + 1);
      }
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        if (j + q < kRun && m + 32 * q < n) {
          const int64_t len = en[q] - st[q];
          if (len > kShortMax) {
            const int key = bucket_of_packets((len + 31) >> 5);
            if (key != run_key) {
              if (same != 0) atomicAdd(&h[run_key], same);
              run_key = key;
              same = 0;
            }
            ++same;
          } else {
            ++short_count;
          }
        }
      }
    }
    advance();
    m = run + lane;
    j = 0;
  }
  if (same != 0) atomicAdd(&h[run_key], same);
  // Bucket 2, one shared atomic per warp; then the block's histogram goes
  // to hist, one global atomic per non-empty bucket.
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) short_count += __shfl_xor_sync(0xffffffffu, short_count, d);
  if (lane == 0 && short_count != 0) atomicAdd(&h[2], short_count);
  __syncthreads();
  for (int i = tid; i < kBuckets; i += 256)
    if (h[i] != 0) atomicAdd(&hist[i], h[i]);
}

template <int W, int NST, int WARPS, bool kHuge>
cudaError_t launch_ragged_v(const Batch& b, const Queue& q, int num_sms, cudaStream_t stream) {
  using L = RaggedLayout<W, NST>;
  constexpr int kBytes = WARPS * L::kWarpBytes;
  auto kern = ragged_kernel<W, NST, WARPS, kHuge>;
  cudaError_t e;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), WARPS * 32, kBytes, &e);
  if (e != cudaSuccess) return e;
  const int64_t blocks_needed = (q.tiles + WARPS - 1) / WARPS;
  const int64_t cap = static_cast<int64_t>(per_sm) * num_sms;
  const int grid = static_cast<int>(blocks_needed < cap ? blocks_needed : cap);
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, WARPS * 32, kBytes, stream>>>(b, q);
  return cudaGetLastError();
}

// Large sorted batches (q.skip_if_short): the variant without the
// huge-message phase, then the one with it; one of the two returns at once.
// Otherwise the variant with the phase alone.
template <int W, int NST, int WARPS>
cudaError_t launch_ragged_t(const Batch& b, const Queue& q, int num_sms, cudaStream_t stream) {
  if (q.skip_if_short) {
    const cudaError_t e = launch_ragged_v<W, NST, WARPS, false>(b, q, num_sms, stream);
    if (e != cudaSuccess) return e;
  }
  return launch_ragged_v<W, NST, WARPS, true>(b, q, num_sms, stream);
}

}  // namespace

cudaError_t launch_short(const Batch& b, const int* run_if, int num_sms, cudaStream_t stream) {
  void (*kern)(Batch, const int*) = b.stream_mode != kWholeMessages ? short_kernel<true, 0>
                                    : b.words == 1                 ? short_kernel<false, 1>
                                    : b.words == 2                 ? short_kernel<false, 2>
                                                                   : short_kernel<false, 4>;
  cudaError_t e;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), 256, 0, &e);
  if (e != cudaSuccess) return e;
  // At least one full wave, and at most 64 messages per thread: with one
  // wave and a fixed share per thread, the blocks the scheduler favoured
  // finished early and left SMs short of warps (a 2^26-message batch with a
  // key per message: 31.9 against 35.0 G hashes/s); later waves fill in.
  const int64_t blocks = (b.n + 255) / 256;
  const int64_t wave = static_cast<int64_t>(per_sm) * num_sms;
  const int64_t cap = wave > (b.n + 256 * 64 - 1) / (256 * 64) ? wave : (b.n + 256 * 64 - 1) / (256 * 64);
  const int grid = static_cast<int>(blocks < cap ? blocks : cap);
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, 256, 0, stream>>>(b, run_if);
  return cudaGetLastError();
}

cudaError_t launch_short_counted(const Batch& b, uint32_t* hist, int num_sms,
                                 cudaStream_t stream) {
  void (*kern)(Batch, uint32_t*) = b.words == 1   ? short_count_kernel<1>
                                   : b.words == 2 ? short_count_kernel<2>
                                                  : short_count_kernel<4>;
  cudaError_t e;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), 256, 0, &e);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (b.n + kCountWarps * kRunMsgs - 1) / (kCountWarps * kRunMsgs);
  const int64_t cap = static_cast<int64_t>(per_sm) * num_sms;
  const int grid = static_cast<int>(blocks < cap ? blocks : cap);
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, kCountWarps * 32, 0, stream>>>(b, hist);
  return cudaGetLastError();
}

bool ragged_shape_valid(StagedShape shape) {
#define HH_VALID(W_, N_) \
  if (shape.window == W_ && shape.stages == N_) return true;
  HH_RAGGED_SHAPES(HH_VALID)
#undef HH_VALID
  return false;
}

cudaError_t launch_ragged(const Batch& b, const Queue& q, StagedShape shape, int num_sms,
                          cudaStream_t stream) {
#define HH_RAGGED(W_, N_) \
  if (shape.window == W_ && shape.stages == N_) return launch_ragged_t<W_, N_, kRaggedWarps>(b, q, num_sms, stream);
  HH_RAGGED_SHAPES(HH_RAGGED)
#undef HH_RAGGED
  return cudaErrorInvalidValue;
}

}  // namespace hh
