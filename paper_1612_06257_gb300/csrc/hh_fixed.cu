// hh_fixed.cu -- fixed-length batches through 2D tensor-map TMA loads.
//
// A batch of n messages of `len` bytes (len a multiple of 16, 16-byte aligned
// base) is a 2D byte tensor [n][len].  A CTA of 128 threads owns tiles of 128
// consecutive messages (one thread per message, the 1024-bit state in
// registers).  For each W-byte window of the tile one thread issues W/128
// tensor loads of a 128-row x 128-byte box (128-byte swizzle) into a shared
// memory stage; NST stages form a ring guarded by "full" mbarriers (TMA
// transaction bytes) and "empty" mbarriers (one arrival per warp once it has
// read the stage).  The stream of (tile, window) pairs runs on across tiles,
// so the next tile's first windows load while the current one finishes.
//
// Thread t reads its 32-byte packets from row t of the box: 16-byte chunk c
// lies at chunk position c ^ (t & 7), so the 8 threads of a quarter-warp hit
// 8 distinct chunks (all 32 banks) on every 128-bit shared load.  Bytes past
// the end of a message and rows past the end of the batch are zero-filled by
// the TMA unit; they are never hashed.
//
// Giving up (a barrier wait that runs past its limit) stops that thread's
// waiting and hashing (it writes zero hashes).  Three rules keep the
// pipeline sound afterwards:
//  - a warp arrives on an "empty" barrier only while its lane 0 is still
//    live.  The lanes of a warp meet at __syncwarp every step, so a warp can
//    run ahead of the real phases only once lane 0 has stopped waiting, and
//    from then on it no longer arrives: every arrival means that warp has
//    finished reading the buffer, and a refill never overwrites data in use
//    (a warp that stops arriving makes the producer's next "empty" wait run
//    out, which ends the refills);
//  - thread 0 refills a buffer only after its own wait for the buffer's
//    previous load succeeded, so at most one load per buffer is in flight
//    and no "full" phase is armed twice; after an "empty" wait that ran out
//    it issues nothing more;
//  - before the CTA exits, thread 0 works out from its cursor how many loads
//    it issued and waits (kDrainLimitNs each) for those it did not see land,
//    load q on buffer q mod NST at phase parity (q / NST) mod 2: at most one
//    per buffer is outstanding and every earlier phase of its buffer has
//    completed, so the parity names the phase.  No bulk copy is in flight
//    when the CTA's shared memory is released.
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
  static constexpr int kBytes = kBarOffset + 2 * NST * 8 + 1024;  // + alignment slack
};

__device__ __forceinline__ void load_swizzled_packet(const uint8_t* box, int row, int chunk,
                                                     uint32_t w[8]) {
  const uint8_t* r = box + row * 128;
  const uint4 a = lds128(r + (((chunk) ^ (row & 7)) << 4));
  const uint4 b = lds128(r + (((chunk + 1) ^ (row & 7)) << 4));
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}

// Thread 0, before the CTA exits: `issued` loads went out (load q into buffer
// q mod nst, completing phase q / nst), and it saw loads 0 .. stop_g - 1 land
// (stop_g < 0: all of them); wait for the others.
__device__ __forceinline__ void drain_loads(uint64_t* full, int nst, int64_t issued,
                                            int64_t stop_g) {
  for (int64_t q = stop_g < 0 ? issued : stop_g; q < issued; ++q)
    mbar_wait_bounded(&full[q % nst], static_cast<uint32_t>((q / nst) & 1), kDrainLimitNs);
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
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
  uint64_t* empty = full + NST;

  const int t = threadIdx.x, lane = t & 31;
  const int64_t steps = (p.len + W - 1) / W;                 // windows per message (>= 1)
  const int64_t tiles = (p.n + kTileMsgs - 1) / kTileMsgs;
  const int64_t my_tiles = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * steps;                    // this CTA's (tile, window) stream

  if (t == 0) {
    prefetch_tensormap(&tmap);
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kRows / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();

  // Producer cursor (thread 0 only): the (tile, window) of the next load.
  int64_t p_tile = blockIdx.x, p_k = 0;
  int p_buf = 0;
  auto issue_next = [&]() {
    mbar_arrive_expect_tx(&full[p_buf], L::kStageBytes);
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int x = 0; x < kBoxes; ++x)
        tma_load_2d(smem + p_buf * L::kStageBytes + (i * kBoxes + x) * kBoxBytes, &tmap,
                    static_cast<int32_t>(p_k * W) + 128 * x,
                    static_cast<int32_t>(p_tile * kTileMsgs + i * kRows), &full[p_buf]);
    if (++p_k == steps) {
      p_k = 0;
      p_tile += gridDim.x;
    }
    p_buf = (p_buf + 1 == NST) ? 0 : p_buf + 1;
  };
  if (t == 0)
    for (int64_t g = 0; g < NST && g < total; ++g) issue_next();

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
  int64_t stop_g = -1;   // thread 0: the step at which it gave up (-1: never)
  bool stopped = false;  // thread 0: an "empty" wait ran out; no further loads
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
        if (t == 0) stop_g = g;
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
      if (lane == 0 && ok) mbar_arrive(&empty[b]);
      if (t == 0 && ok && !stopped && g + NST < total) {
        // Refill this buffer once every warp has read it.
        if (!mbar_wait_bounded(&empty[b], parity, limit)) {
          record_error(p.err, kErrTimeout);
          stopped = true;  // refills stop for good: the cursor must stay in step
        } else {
          fence_proxy_async_smem();
          issue_next();
        }
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
  // Loads issued but never waited for (only after a timeout) get a bounded
  // time to land before the CTA exits.
  if (t == 0) drain_loads(full, NST, (p_tile - blockIdx.x) / gridDim.x * steps + p_k, stop_g);
}

// Two threads per message, for batches too small to fill the GPU: threads
// 2r and 2r + 1 keep lane pairs (0, 1) and (2, 3) of row r's state (Update
// mixes lanes only within a pair), so each thread's Update chain is half
// as long; they trade v0 in finalisation.  Tiles of ROWS messages (32, 64
// or 128: the launcher picks the largest that still gives every SM a tile)
// with the same windows and full/empty barrier protocol as fixed_tma_kernel.
template <int W, int NST, int ROWS>
struct PairLayout {
  static constexpr int kBoxBytes = 128 * ROWS;
  static constexpr int kStageBytes = W * ROWS;
  static constexpr int kBarOffset = NST * kStageBytes;
  static constexpr int kBytes = kBarOffset + 2 * NST * 8 + 1024;  // + alignment slack
};

template <int W, int NST, int ROWS, bool kCustom>
__global__ void __launch_bounds__(2 * ROWS) fixed_pair_kernel(
    const __grid_constant__ CUtensorMap tmap, FixedParams p) {
  const uint64_t limit = kCustom ? p.wait_ns : kWaitLimitNs;
  using L = PairLayout<W, NST, ROWS>;
  constexpr int kBoxes = W / 128;
  constexpr int kWarps = 2 * ROWS / 32;
  constexpr int kBoxB = L::kBoxBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
  uint64_t* empty = full + NST;

  const int t = threadIdx.x, lane = t & 31, row = t >> 1, half = t & 1;
  const int64_t steps = (p.len + W - 1) / W;
  const int64_t tiles = (p.n + ROWS - 1) / ROWS;
  const int64_t my_tiles = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * steps;

  if (t == 0) {
    prefetch_tensormap(&tmap);
    for (int i = 0; i < NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  int64_t p_tile = blockIdx.x, p_k = 0;
  int p_buf = 0;
  auto issue_next = [&]() {
    mbar_arrive_expect_tx(&full[p_buf], L::kStageBytes);
#pragma unroll
    for (int x = 0; x < kBoxes; ++x)
      tma_load_2d(smem + p_buf * L::kStageBytes + x * kBoxB, &tmap,
                  static_cast<int32_t>(p_k * W) + 128 * x, static_cast<int32_t>(p_tile * ROWS),
                  &full[p_buf]);
    if (++p_k == steps) {
      p_k = 0;
      p_tile += gridDim.x;
    }
    p_buf = (p_buf + 1 == NST) ? 0 : p_buf + 1;
  };
  if (t == 0)
    for (int64_t g = 0; g < NST && g < total; ++g) issue_next();

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
  int64_t stop_g = -1;   // thread 0: the step at which it gave up (-1: never)
  bool stopped = false;  // thread 0: an "empty" wait ran out; no further loads
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
        if (t == 0) stop_g = g;
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
      if (lane == 0 && ok) mbar_arrive(&empty[b]);
      if (t == 0 && ok && !stopped && g + NST < total) {
        if (!mbar_wait_bounded(&empty[b], parity, limit)) {
          record_error(p.err, kErrTimeout);
          stopped = true;  // refills stop for good: the cursor must stay in step
        } else {
          fence_proxy_async_smem();
          issue_next();
        }
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
  if (t == 0) drain_loads(full, NST, (p_tile - blockIdx.x) / gridDim.x * steps + p_k, stop_g);
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
