// hh_fixed.cu -- fixed-length batches through 2D tensor-map TMA loads.
//
// A batch of n messages of `len` bytes (len a multiple of 16, 16-byte aligned
// base) is a 2D byte tensor [n][len].  A CTA of 128 threads owns tiles of 128
// consecutive messages (one thread per message, the 1024-bit state in
// registers).  Each W-byte window of the tile is W/128 tensor loads of a
// 128-row x 128-byte box (128-byte swizzle) into a shared-memory stage; NST
// stages form a ring, each with a "full" mbarrier (TMA transaction bytes).
// The stream of (tile, window) pairs runs on across tiles, so the next
// tile's first windows load while the current one finishes.
//
// Thread t reads its 32-byte packets from row t of the box: 16-byte chunk c
// lies at chunk position c ^ (t & 7), so the 8 threads of a quarter-warp hit
// 8 distinct chunks (all 32 banks) on every 128-bit shared load.  Bytes past
// the end of a message and rows past the end of the batch are zero-filled by
// the TMA unit; they are never hashed.
//
// The last warp to finish reading a stage refills it.  Once a warp's lanes
// have read the stage (they meet at __syncwarp), lane 0 bumps the stage's
// "done" counter with an acquire-release increment that wraps at the warp
// count; the warp whose increment completes the count issues the load of
// window g + NST into the stage.  No thread waits for the others to finish
// with a stage, only for its data to land.
//
// Giving up (a "full" wait that runs past its limit) stops that thread's
// waiting and hashing (it writes zero hashes).  Two rules keep the pipeline
// sound afterwards:
//  - a warp counts itself done only while its lane 0 is live.  A lane that
//    gave up reads no shared memory again, so every count means that warp
//    has finished with the stage and a refill never overwrites data in use.
//    A warp whose lane 0 gave up never counts again: no stage is refilled
//    after that, and the other warps' waits run out in turn.  A stage's next
//    load goes out only after every warp saw its previous load land, so at
//    most one load per stage is in flight and no "full" phase is armed twice;
//  - the issuer records how many loads went into the stage.  Before the CTA
//    exits all threads meet, and thread b waits (kDrainLimitNs) for the last
//    load into stage b at the parity of its number: every earlier load into
//    that stage has completed, so the parity names the phase.  No bulk copy
//    is in flight when the CTA's shared memory is released.
// The limit is a compile-time 2 s in the kernels every call uses; a context
// with its own limit (hh_set_tune_param "wait_limit_ns") runs separate
// instantiations that read it from their parameters.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "hh_device.cuh"
#include "hh_internal.h"
#include "hh_ptx.cuh"

namespace hh {
namespace {

constexpr int kRows = 128;           // messages per tile = box height = threads
constexpr int kBoxBytes = 128 * kRows;

struct FixedParams {
  int64_t n;
  int64_t len;
  const uint64_t* keys;
  int per_message_keys;
  uint64_t* out;
  int words;
  int* err;
  uint32_t one;
  uint64_t wait_ns;  // the context's wait limit (read by the kCustom kernels only)
};

template <int W, int NST, int M>
struct FixedLayout {
  static constexpr int kStageBytes = W * kRows * M;
  static constexpr int kBarOffset = NST * kStageBytes;
  static constexpr int kBytes = kBarOffset + NST * 8 + 2 * NST * 4 + 1024;  // + counters, slack
};

__device__ __forceinline__ void load_swizzled_packet(const uint8_t* box, int row, int chunk,
                                                     uint32_t w[8]) {
  const uint8_t* r = box + row * 128;
  const uint4 a = lds128(r + (((chunk) ^ (row & 7)) << 4));
  const uint4 b = lds128(r + (((chunk + 1) ^ (row & 7)) << 4));
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}

// The (tile, window) `ahead` windows after (tile, k) in this CTA's stream of
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... of `steps` windows each.
__device__ __forceinline__ void advance(int64_t& tile, int64_t& k, int ahead, int64_t steps) {
  k += ahead;
  while (k >= steps) {
    k -= steps;
    tile += gridDim.x;
  }
}

// The shared-memory words beside the "full" barriers: per stage the warps
// done with its current load, and the number of loads issued into it.
struct RingCounters {
  uint32_t* done;
  uint32_t* loads;
};

__device__ __forceinline__ RingCounters ring_counters(uint64_t* full, int nst) {
  uint32_t* w = reinterpret_cast<uint32_t*>(full + nst);
  return {w, w + nst};
}

// Every thread, before the CTA exits: thread b < nst waits (bounded) for the
// last load issued into stage b, the only one that can still be in flight.
__device__ __forceinline__ void drain_last_loads(uint64_t* full, RingCounters c, int nst, int t) {
  __syncthreads();
  if (t < nst && c.loads[t] > 0)
    mbar_wait_bounded(&full[t], (c.loads[t] - 1) & 1u, kDrainLimitNs);
}

// M messages per thread: a tile is 128 * M messages; thread t hashes
// messages t, t + 128, ... of the tile, interleaving M independent Update
// chains for more instruction-level parallelism per warp.
template <int W, int NST, int M, bool kCustom>
__global__ void __launch_bounds__(kRows) fixed_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                          FixedParams p) {
  const uint64_t limit = kCustom ? p.wait_ns : kWaitLimitNs;
  using L = FixedLayout<W, NST, M>;
  constexpr int kBoxes = W / 128;
  constexpr int kTileMsgs = kRows * M;
  constexpr uint32_t kWarps = kRows / 32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
  const RingCounters ring = ring_counters(full, NST);

  const int t = threadIdx.x, lane = t & 31;
  const int64_t steps = (p.len + W - 1) / W;                 // windows per message (>= 1)
  const int64_t tiles = (p.n + kTileMsgs - 1) / kTileMsgs;
  const int64_t my_tiles = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * steps;                    // this CTA's (tile, window) stream

  auto issue = [&](int64_t ltile, int64_t lk, int buf) {
    mbar_arrive_expect_tx(&full[buf], L::kStageBytes);
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int x = 0; x < kBoxes; ++x)
        tma_load_2d(smem + buf * L::kStageBytes + (i * kBoxes + x) * kBoxBytes, &tmap,
                    static_cast<int32_t>(lk * W) + 128 * x,
                    static_cast<int32_t>(ltile * kTileMsgs + i * kRows), &full[buf]);
  };
  if (t == 0) {
    prefetch_tensormap(&tmap);
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      ring.done[i] = 0;
      ring.loads[i] = 0;
    }
    fence_mbar_init();
    int64_t lt = blockIdx.x, lk = 0;
    for (int q = 0; q < NST && q < total; ++q) {
      ring.loads[q] = 1;
      issue(lt, lk, q);
      advance(lt, lk, 1, steps);
    }
  }
  __syncthreads();

  const int64_t packets = p.len >> 5;
  const uint32_t r = static_cast<uint32_t>(p.len & 31);
  const int64_t rem_step = r ? (packets * 32) / W : -1;
  const int rem_off = r ? static_cast<int>(packets * 32 - rem_step * W) : 0;
  uint64_t key[4];
  if (!p.per_message_keys) {
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = __ldg(p.keys + i);
  }
  State s[M];
  bool ok = true;
  int b = 0;                // stage buffer of the current window
  uint32_t parity = 0;      // its phase parity
  int64_t g = 0;            // position in this CTA's (tile, window) stream
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t m0 = tile * kTileMsgs + t;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      if (p.per_message_keys) {
        const int64_t m = m0 + i * kRows;
        const uint64_t* kp = p.keys + 4 * (m < p.n ? m : 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) key[q] = __ldg(kp + q);
      }
      init(s[i], key);
    }
    for (int64_t k = 0; k < steps; ++k, ++g) {
      if (ok && !mbar_wait_bounded(&full[b], parity, limit)) {
        ok = false;
        record_error(p.err, kErrTimeout);
      }
      const uint8_t* stage = smem + b * L::kStageBytes;
      if (ok) {
        const int64_t p0 = k * (W / 32);
#pragma unroll
        for (int j = 0; j < W / 32; ++j) {
          if (p0 + j < packets) {
#pragma unroll
            for (int i = 0; i < M; ++i) {
              uint32_t w[8];
              load_swizzled_packet(stage + (i * kBoxes + j / 4) * kBoxBytes, t, (j % 4) * 2, w);
              update_words_v<kFastUpdate>(s[i], w, p.one);
            }
          }
        }
        if (k == rem_step) {
#pragma unroll
          for (int i = 0; i < M; ++i) {
            uint32_t w[8];
            load_swizzled_packet(stage + (i * kBoxes + rem_off / 128) * kBoxBytes, t,
                                 (rem_off % 128) / 16, w);
            remainder(s[i], r, w);
          }
        }
      }
      __syncwarp();
      // The last warp done with this stage loads window g + NST into it.
      if (lane == 0 && ok && atom_inc_wrap_acq_rel(&ring.done[b], kWarps - 1) == kWarps - 1 &&
          g + NST < total) {
        int64_t lt = tile, lk = k;
        advance(lt, lk, NST, steps);
        ring.loads[b] = static_cast<uint32_t>((g + NST) / NST + 1);
        fence_proxy_async_smem();
        issue(lt, lk, b);
      }
      if (++b == NST) {
        b = 0;
        parity ^= 1u;
      }
    }
#pragma unroll
    for (int i = 0; i < M; ++i) finalize(s[i]);
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int64_t m = m0 + i * kRows;
      if (m < p.n) {
        uint64_t h[4];
        digest(s[i], h);
        if (!ok) h[0] = h[1] = h[2] = h[3] = 0;
        uint64_t* o = p.out + m * p.words;
        o[0] = h[0];
        if (p.words >= 2) o[1] = h[1];
        if (p.words == 4) {
          o[2] = h[2];
          o[3] = h[3];
        }
      }
    }
  }
  drain_last_loads(full, ring, NST, t);
}

// Two threads per message, for batches too small to fill the GPU: threads
// 2r and 2r + 1 keep lane pairs (0, 1) and (2, 3) of row r's state (Update
// mixes lanes only within a pair), so each thread's Update chain is half
// as long; they trade v0 in finalisation.  Tiles of ROWS messages (32, 64
// or 128: the launcher picks the largest that still gives every SM a tile)
// with the same windows and stage ring protocol as fixed_tma_kernel.
template <int W, int NST, int ROWS>
struct PairLayout {
  static constexpr int kBoxBytes = 128 * ROWS;
  static constexpr int kStageBytes = W * ROWS;
  static constexpr int kBarOffset = NST * kStageBytes;
  static constexpr int kBytes = kBarOffset + NST * 8 + 2 * NST * 4 + 1024;  // + counters, slack
};

template <int W, int NST, int ROWS, bool kCustom>
__global__ void __launch_bounds__(2 * ROWS) fixed_pair_kernel(
    const __grid_constant__ CUtensorMap tmap, FixedParams p) {
  const uint64_t limit = kCustom ? p.wait_ns : kWaitLimitNs;
  using L = PairLayout<W, NST, ROWS>;
  constexpr int kBoxes = W / 128;
  constexpr uint32_t kWarps = 2 * ROWS / 32;
  constexpr int kBoxB = L::kBoxBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
  const RingCounters ring = ring_counters(full, NST);

  const int t = threadIdx.x, lane = t & 31, row = t >> 1, half = t & 1;
  const int64_t steps = (p.len + W - 1) / W;
  const int64_t tiles = (p.n + ROWS - 1) / ROWS;
  const int64_t my_tiles = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * steps;

  auto issue = [&](int64_t ltile, int64_t lk, int buf) {
    mbar_arrive_expect_tx(&full[buf], L::kStageBytes);
#pragma unroll
    for (int x = 0; x < kBoxes; ++x)
      tma_load_2d(smem + buf * L::kStageBytes + x * kBoxB, &tmap,
                  static_cast<int32_t>(lk * W) + 128 * x, static_cast<int32_t>(ltile * ROWS),
                  &full[buf]);
  };
  if (t == 0) {
    prefetch_tensormap(&tmap);
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      ring.done[i] = 0;
      ring.loads[i] = 0;
    }
    fence_mbar_init();
    int64_t lt = blockIdx.x, lk = 0;
    for (int q = 0; q < NST && q < total; ++q) {
      ring.loads[q] = 1;
      issue(lt, lk, q);
      advance(lt, lk, 1, steps);
    }
  }
  __syncthreads();

  const int64_t packets = p.len >> 5;
  const uint32_t r = static_cast<uint32_t>(p.len & 31);
  const int64_t rem_step = r ? (packets * 32) / W : -1;
  const int rem_off = r ? static_cast<int>(packets * 32 - rem_step * W) : 0;
  uint64_t key[4];
  if (!p.per_message_keys) {
#pragma unroll
    for (int i = 0; i < 4; ++i) key[i] = __ldg(p.keys + i);
  }
  Half s;
  bool ok = true;
  int b = 0;
  uint32_t parity = 0;
  int64_t g = 0;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t m = tile * ROWS + row;
    if (p.per_message_keys) {
      const uint64_t* kp = p.keys + 4 * (m < p.n ? m : 0);
#pragma unroll
      for (int q = 0; q < 4; ++q) key[q] = __ldg(kp + q);
    }
    init_half(s, key, half);
    for (int64_t k = 0; k < steps; ++k, ++g) {
      if (ok && !mbar_wait_bounded(&full[b], parity, limit)) {
        ok = false;
        record_error(p.err, kErrTimeout);
      }
      const uint8_t* stage = smem + b * L::kStageBytes;
      if (ok) {
        const int64_t p0 = k * (W / 32);
#pragma unroll
        for (int j = 0; j < W / 32; ++j) {
          if (p0 + j < packets) {
            const uint8_t* rp = stage + (j / 4) * kBoxB + row * 128;
            const uint4 a = lds128(rp + ((((j % 4) * 2 + half) ^ (row & 7)) << 4));
            update_half(s, join(a.x, a.y), join(a.z, a.w));
          }
        }
        if (k == rem_step) {
          uint32_t w[8], pk[8];
          load_swizzled_packet(stage + (rem_off / 128) * kBoxB, row, (rem_off % 128) / 16, w);
          remainder_packet(r, w, pk);
          inject_size_half(s, r);
          if (half == 0) update_half(s, join(pk[0], pk[1]), join(pk[2], pk[3]));
          else update_half(s, join(pk[4], pk[5]), join(pk[6], pk[7]));
        }
      }
      __syncwarp();
      if (lane == 0 && ok && atom_inc_wrap_acq_rel(&ring.done[b], kWarps - 1) == kWarps - 1 &&
          g + NST < total) {
        int64_t lt = tile, lk = k;
        advance(lt, lk, NST, steps);
        ring.loads[b] = static_cast<uint32_t>((g + NST) / NST + 1);
        fence_proxy_async_smem();
        issue(lt, lk, b);
      }
      if (++b == NST) {
        b = 0;
        parity ^= 1u;
      }
    }
    finalize_half(s);
    if (m < p.n) {
      const uint64_t keep = ok ? ~0ull : 0ull;
      const uint64_t h0 = (s.v0[0] + s.v1[0] + s.mul0[0] + s.mul1[0]) & keep;
      const uint64_t h1 = (s.v0[1] + s.v1[1] + s.mul0[1] + s.mul1[1]) & keep;
      uint64_t* o = p.out + m * p.words;
      if (half == 0) {
        o[0] = h0;
        if (p.words >= 2) o[1] = h1;
      } else if (p.words == 4) {
        o[2] = h0;
        o[3] = h1;
      }
    }
  }
  drain_last_loads(full, ring, NST, t);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

template <int W, int NST, int M>
cudaError_t launch_fixed_t(const CUtensorMap& tmap, const FixedParams& p, int num_sms,
                           cudaStream_t stream) {
  using L = FixedLayout<W, NST, M>;
  auto kern = p.wait_ns == kWaitLimitNs ? fixed_tma_kernel<W, NST, M, false>
                                        : fixed_tma_kernel<W, NST, M, true>;
  cudaError_t e;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), kRows, L::kBytes, &e);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (p.n + kRows * M - 1) / (kRows * M);
  const int64_t cap = static_cast<int64_t>(per_sm) * num_sms;
  const int grid = static_cast<int>(tiles < cap ? tiles : cap);
  kern<<<grid, kRows, L::kBytes, stream>>>(tmap, p);
  return cudaGetLastError();
}

}  // namespace

bool fixed_tma_supported(const uint8_t* bytes, int64_t len, int64_t n) {
  return encode_fn() != nullptr && len > 0 && len % 16 == 0 &&
         (reinterpret_cast<uintptr_t>(bytes) % 16) == 0 && n > 0 && n < (int64_t(1) << 31) &&
         len < (int64_t(1) << 31);
}

bool fixed_shape_valid(StagedShape shape) {
#define HH_VALID(W_, N_, M_) \
  if (shape.window == W_ && shape.stages == N_ && shape.msgs == M_) return true;
  HH_FIXED_SHAPES(HH_VALID)
#undef HH_VALID
  return false;
}

template <int W, int NST, int ROWS>
cudaError_t launch_fixed_pair_t(const CUtensorMap& tmap, const FixedParams& p, int num_sms,
                                cudaStream_t stream) {
  using L = PairLayout<W, NST, ROWS>;
  auto kern = p.wait_ns == kWaitLimitNs ? fixed_pair_kernel<W, NST, ROWS, false>
                                        : fixed_pair_kernel<W, NST, ROWS, true>;
  cudaError_t e;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), 2 * ROWS, L::kBytes, &e);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (p.n + ROWS - 1) / ROWS;
  const int64_t cap = static_cast<int64_t>(per_sm) * num_sms;
  const int grid = static_cast<int>(tiles < cap ? tiles : cap);
  kern<<<grid, 2 * ROWS, L::kBytes, stream>>>(tmap, p);
  return cudaGetLastError();
}

namespace {

// The batch as a 2D tensor [n][len] of bytes, loaded in `rows`-row x
// 128-byte boxes with the 128-byte swizzle.
cudaError_t encode_rows(const Batch& b, CUtensorMap* tmap, int rows) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(b.fixed_len), static_cast<cuuint64_t>(b.n)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(b.fixed_len)};
  const cuuint32_t box[2] = {128, static_cast<cuuint32_t>(rows)};
  const cuuint32_t elem[2] = {1, 1};
  CUresult r = enc(tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(b.bytes), dims,
                   strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fixed_tma(const Batch& b, StagedShape shape, int num_sms,
                             cudaStream_t stream) {
  CUtensorMap tmap;
  cudaError_t e = encode_rows(b, &tmap, kRows);
  if (e != cudaSuccess) return e;
  FixedParams p{b.n, b.fixed_len, b.keys, b.per_message_keys, b.out, b.words, b.err, 1u,
                b.wait_ns};
#define HH_FIXED(W_, N_, M_)                                          \
  if (shape.window == W_ && shape.stages == N_ && shape.msgs == M_) \
    return launch_fixed_t<W_, N_, M_>(tmap, p, num_sms, stream);
  HH_FIXED_SHAPES(HH_FIXED)
#undef HH_FIXED
  return cudaErrorInvalidValue;
}

cudaError_t launch_fixed_tma_pair(const Batch& b, int num_sms, cudaStream_t stream) {
  // The largest tile height that still gives every SM a tile.
  const int rows = b.n >= 128 * static_cast<int64_t>(num_sms)  ? 128
                   : b.n >= 64 * static_cast<int64_t>(num_sms) ? 64
                                                              : 32;
  CUtensorMap tmap;
  cudaError_t e = encode_rows(b, &tmap, rows);
  if (e != cudaSuccess) return e;
  FixedParams p{b.n, b.fixed_len, b.keys, b.per_message_keys, b.out, b.words, b.err, 1u,
                b.wait_ns};
  if (rows == 128) return launch_fixed_pair_t<256, 2, 128>(tmap, p, num_sms, stream);
  if (rows == 64) return launch_fixed_pair_t<256, 2, 64>(tmap, p, num_sms, stream);
  return launch_fixed_pair_t<256, 2, 32>(tmap, p, num_sms, stream);
}

}  // namespace hh
