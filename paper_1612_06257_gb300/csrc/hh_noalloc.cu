// hh_noalloc.cu -- a ragged-batch hash call that allocates no memory.
//
// Some callers cannot allocate device memory for this library: their device
// memory is owned by another allocator (a framework's caching pool or a fixed
// memory budget that out-of-band cudaMalloc would break), or they sit on a
// latency-critical path where cudaMalloc's implicit device synchronisation is
// not acceptable.  hh_hash_batch_noalloc serves them.  It runs the same
// length sort and warp-tile kernel as hh_hash{64,128,256}_batch, but the
// sort's scratch (message order, bucket counts and cursors, the work-queue
// counter, a flag and a spare error word) lives in one file-scope __device__
// array of fixed size, which every GPU that loads the library holds until
// the process exits.  The caller still passes all inputs and outputs.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "hh.h"
#include "hh_internal.h"

namespace {

constexpr int64_t kMaxMessages = HH_NOALLOC_MAX_MESSAGES;
constexpr int kMaxDevices = 64;

struct Scratch {
  int32_t perm[kMaxMessages];
  uint32_t hist[hh::kBuckets];
  uint32_t cursor[hh::kBuckets];
  unsigned long long next_tile[4];
  long long huge_count;
  int use_perm;
  int err;
};

// The shared scratch.  In host code this name is only a stand-in for the
// symbol; kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[sizeof(Scratch)];

struct DeviceSlot {
  bool ready = false;
  Scratch* scratch = nullptr;  // device address of g_scratch on this device
  int num_sms = 0;
};

std::mutex g_mutex;
DeviceSlot g_slots[kMaxDevices];

// Once per device, with that device current: look up the scratch address.
int slot_for_current_device(DeviceSlot** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HH_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) return HH_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      return HH_ERR_CUDA;
    s.scratch = static_cast<Scratch*>(ptr);
    s.num_sms = sms;
    s.ready = true;
  }
  *out = &s;
  return HH_OK;
}

}  // namespace

extern "C" int hh_hash_batch_noalloc(int bits, const uint64_t* keys, int key_mode,
                                     const uint8_t* bytes, const int64_t* offsets, int64_t n,
                                     uint64_t* out, int* device_error, void* stream) {
  const int words = bits == 64 ? 1 : bits == 128 ? 2 : bits == 256 ? 4 : 0;
  if (words == 0 || (key_mode != HH_KEY_SHARED && key_mode != HH_KEY_PER_MESSAGE) || n < 0)
    return HH_ERR_INVALID_ARG;
  if (n > kMaxMessages) return HH_ERR_TOO_LARGE;
  if (n == 0) return HH_OK;
  if (keys == nullptr || bytes == nullptr || offsets == nullptr || out == nullptr)
    return HH_ERR_INVALID_ARG;
  DeviceSlot* slot = nullptr;
  const int st = slot_for_current_device(&slot);
  if (st != HH_OK) return st;
  Scratch* scr = slot->scratch;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  hh::Batch b{};
  b.bytes = bytes;
  b.offsets = offsets;
  b.fixed_len = 0;
  b.seg_start = nullptr;
  b.keys = keys;
  b.per_message_keys = key_mode == HH_KEY_PER_MESSAGE;
  b.n = n;
  b.out = out;
  b.words = words;
  b.err = device_error ? device_error : &scr->err;

  // The sort clears the bucket counts itself and its scan resets the queue
  // counter and the flag, so nothing left by an earlier call is read.
  int launches = 0;
  cudaError_t e = hh::launch_bucket_sort(b, scr->hist, scr->cursor, scr->perm,
                                         scr->next_tile, &scr->use_perm, &scr->huge_count,
                                         hh::kHugeBucket, slot->num_sms, s, &launches);
  if (e != cudaSuccess) return HH_ERR_CUDA;
  hh::Queue q{};
  q.perm = scr->perm;
  q.use_perm = &scr->use_perm;
  q.huge_count = &scr->huge_count;
  q.next_tile = scr->next_tile;
  q.solo_max = static_cast<int64_t>(hh::kSoloPerSm) * slot->num_sms;
  q.solo_ctas = static_cast<int>((q.solo_max + hh::kRaggedWarps - 1) / hh::kRaggedWarps);
  q.tiles = (n + 31) / 32 > q.solo_max ? (n + 31) / 32 : (n < q.solo_max ? n : q.solo_max);
  e = hh::launch_ragged(b, q, hh::StagedShape{256, 2}, slot->num_sms, s);
  return e == cudaSuccess ? HH_OK : HH_ERR_CUDA;
}
