/*
 * hh.h -- C ABI of libhh, a batched HighwayHash engine for NVIDIA GB300 (sm_103a).
 *
 * HighwayHash is the keyed pseudo-random function of Alakuijala, Cox and
 * Wassenberg, "Fast keyed hash/pseudo-random function using SIMD multiply and
 * permute" (arXiv:1612.06257).  A 256-bit key and a message of any length map
 * to a 64-, 128- or 256-bit hash (Sections 1 and 4.3).  Per message the
 * library runs, entirely in its own CUDA kernels:
 *   Init from the key (Section 4.4) -> one Update per whole 32-byte packet
 *   (Section 4.2, with ZipperMerge of Section 4.1) -> size injection and one
 *   padded Update of the last size mod 32 bytes (Section 4.5) -> four rounds
 *   of Update(Permute(v0)) (Section 4.3) -> h[i] = v0[i]+v1[i]+mul0[i]+mul1[i].
 * The 64-bit hash is h[0], the 128-bit hash (h[0], h[1]), the 256-bit hash
 * h[0..3].  Every message is independent.
 *
 * Details the paper leaves open are fixed as follows: packets and keys are
 * little-endian 64-bit lanes, lane 0 first; the size mod 32 is added to each
 * lane of v0 as one 64-bit add of (r << 32) + r; v1's 32-bit halves are
 * rotated left by r; the last r mod 4 bytes go to packet bytes 28..30; the
 * initialisation constants take pi's first hex words most-significant lane
 * first.  Agreement with any released HighwayHash library is not claimed.
 *
 * Conventions for every call below:
 *  - Unless a function says "host", every pointer is a DEVICE pointer (memory
 *    from cudaMalloc, cudaMallocAsync or a caching allocator on the context's
 *    device).  The caller owns all buffers; they must stay valid until the
 *    work queued on `stream` has finished.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Hash calls are asynchronous: they enqueue work and
 *    return; results are ready when the stream reaches that point.
 *  - Errors the host can detect (null pointers, bad sizes, bad modes) are
 *    returned synchronously and nothing is enqueued.  Errors only the device
 *    can see (decreasing offsets, a pipeline wait that ran out) are recorded
 *    in a per-context device error word; read it with hh_get_device_error.
 *    No call aborts, throws or prints.
 *  - One hh_ctx may be used by one host thread at a time.  Calls on one
 *    context from several threads need external locking.  Concurrent calls
 *    on different streams of one context share its scratch memory and must
 *    not overlap on the device.
 */
#ifndef HH_H
#define HH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hh_ctx hh_ctx;

/* Status codes returned by every call. */
enum hh_status {
  HH_OK = 0,
  HH_ERR_INVALID_ARG = 1,   /* null pointer with n > 0, bad mode, bad bits   */
  HH_ERR_CUDA = 2,          /* a CUDA runtime call failed                     */
  HH_ERR_NO_MEMORY = 3,     /* device or host allocation failed               */
  HH_ERR_TIMEOUT = 4,       /* device: a bounded pipeline wait ran out        */
  HH_ERR_TOO_LARGE = 5,     /* a size beyond what the call supports           */
  HH_ERR_BAD_OFFSETS = 6,   /* device: offsets[i+1] < offsets[i] somewhere    */
  HH_ERR_NO_DEVICE = 7,     /* no usable CUDA device with sm_103a             */
  HH_ERR_BAD_KEY_INDEX = 8, /* device: a key index outside the key table      */
  HH_ERR_BAD_CHUNK = 9      /* device: a stream update chunk of 32k+r bytes   */
};

/* How `keys` is laid out. */
enum hh_key_mode {
  HH_KEY_SHARED = 0,        /* keys = uint64[4]: one key for every message    */
  HH_KEY_PER_MESSAGE = 1    /* keys = uint64[n][4]: key of message i at 4*i   */
};

/* Kernel choice (for benchmarking and tests; HH_KERNEL_AUTO is the product
 * default and picks the staged kernels). */
enum hh_kernel {
  HH_KERNEL_AUTO = 0,
  HH_KERNEL_NAIVE = 1,      /* one thread per message, direct global loads    */
  HH_KERNEL_STAGED = 2,     /* length-sorted warp tiles, cp.async staging     */
  HH_KERNEL_STAGED_UNSORTED = 3, /* the same, messages in index order         */
  HH_KERNEL_STAGED_BULK = 4 /* CTA tiles, one bulk async copy per thread      */
};

/*
 * Create a context on CUDA device `device`.  It owns a small device error
 * word, the work-queue counters and the length sort's scratch memory, sized
 * for HH_DEFAULT_MAX_MESSAGES messages per call (16 MiB; raise it with
 * hh_reserve).  `tune_cache_path` names a tuning table written by
 * hh_tune_save (HH_ERR_INVALID_ARG if it cannot be read), or NULL for the
 * built-in choices measured on GB300.
 * Returns HH_ERR_NO_DEVICE when the device is absent or not sm_103a.
 * The caller's current device is restored before returning.
 */
#define HH_DEFAULT_MAX_MESSAGES (1 << 22)
int hh_init(hh_ctx** out, int device, const char* tune_cache_path);

/* Free everything the context owns.  Waits for its device work first.
 * NULL is accepted and ignored. */
int hh_destroy(hh_ctx* ctx);

/*
 * Size the context's length-sort scratch for batches of up to `max_messages`
 * messages (4 bytes per message; it never shrinks).  The hash calls
 * themselves never allocate or synchronise: a ragged, segments or stream
 * call with more messages than the context has room for returns
 * HH_ERR_TOO_LARGE and enqueues nothing (fixed-length batches need no
 * scratch).  Growing the scratch synchronises the device, so reserve before
 * a latency-critical phase or a stream capture.  HH_ERR_TOO_LARGE above
 * 2^31 - 1 messages.
 */
int hh_reserve(hh_ctx* ctx, int64_t max_messages);

/*
 * Hash a ragged batch (Sections 4.2-4.5).
 *   keys     per key_mode: uint64[4] or uint64[n][4], little-endian lanes.
 *   bytes    concatenated message bytes; message i is
 *            bytes[offsets[i] .. offsets[i+1]).  No alignment requirement;
 *            must not be NULL when n > 0.
 *            The library reads only bytes in [offsets[0], offsets[n]).
 *   offsets  int64[n+1], non-decreasing, offsets[0] >= 0.  A decreasing pair
 *            sets HH_ERR_BAD_OFFSETS on the device and that message's output
 *            words are written as zero.
 *   n        number of messages; n == 0 is a no-op returning HH_OK.
 *   out      uint64[n * words] with words = 1, 2, 4 for 64/128/256 bits;
 *            message i's hash is out[words*i .. words*i + words).
 * Returns HH_OK once the work is enqueued on `stream`.
 */
int hh_hash64_batch(hh_ctx* ctx, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                    const int64_t* offsets, int64_t n, uint64_t* out, void* stream);
int hh_hash128_batch(hh_ctx* ctx, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                     const int64_t* offsets, int64_t n, uint64_t* out, void* stream);
int hh_hash256_batch(hh_ctx* ctx, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                     const int64_t* offsets, int64_t n, uint64_t* out, void* stream);

/*
 * Hash a fixed-length batch: message i is bytes[i*msg_len .. (i+1)*msg_len).
 * Same semantics as the ragged calls without the offsets array.  bits is 64,
 * 128 or 256.  bytes may be NULL only when msg_len == 0.  When bytes is
 * 16-byte aligned and msg_len a multiple of 16, a kernel that needs no
 * realignment runs.
 */
int hh_hash_fixed(hh_ctx* ctx, int bits, const uint64_t* keys, int key_mode,
                  const uint8_t* bytes, int64_t msg_len, int64_t n, uint64_t* out,
                  void* stream);

/*
 * Hash a batch given as segments of one byte buffer, each with its own key
 * from a device key table: the batch descriptor of a request server, where
 * messages of many requests share one launch.
 *   key_table  uint64[key_count][4]; key_index int32[n] picks message i's
 *              row (NULL: every message uses row 0).  An index outside
 *              [0, key_count) sets HH_ERR_BAD_KEY_INDEX on the device and the
 *              message's output words are written as zero.
 *   bytes      a buffer of bytes_len bytes (not NULL); message i is
 *              bytes[starts[i] .. starts[i] + lengths[i]).  Segments may come
 *              in any order and may overlap.  A segment that does not lie in
 *              [0, bytes_len) sets HH_ERR_BAD_OFFSETS and gets zero output.
 *              The library reads only bytes inside [0, bytes_len).
 *   n_device   NULL, or a device int64 holding the message count at run time;
 *              then n is only a capacity (the arrays hold n entries) and
 *              the launch configuration depends on n alone, so one captured
 *              launch serves batches of any size up to n.  Reserve scratch
 *              for n messages (hh_reserve) before capturing.
 *   out        uint64[n * bits/64] as for the ragged calls.
 * Same hash (Sections 4.2-4.5), asynchronous on `stream`.
 */
int hh_hash_segments(hh_ctx* ctx, int bits, const uint64_t* key_table, int32_t key_count,
                     const int32_t* key_index, const uint8_t* bytes, int64_t bytes_len,
                     const int64_t* starts, const int64_t* lengths, int64_t n,
                     const int64_t* n_device, uint64_t* out, void* stream);

/*
 * Host-memory variant of the ragged call: keys, bytes, offsets and out are
 * HOST pointers (pinned memory gives full copy speed; pageable works).  The
 * batch is copied to the device in chunks of at most 128 MiB and 2^20
 * messages, hashed there and copied back, with copies and hashing of
 * consecutive chunks overlapped.  Synchronous: returns after `out` is
 * filled, or, on an error, after every copy it started has finished.  Before
 * a chunk is enqueued its offsets are checked on the host: a decreasing pair
 * returns HH_ERR_BAD_OFFSETS (the hashes of earlier chunks are written, the
 * rest of `out` is not).  Unlike the device calls it owns device staging
 * memory (two chunk slots), which it grows on the first call that needs
 * more; the growth is stream-ordered on the context's own copy stream and
 * waits for no other work on the device.  bits is 64, 128 or 256.
 */
int hh_hash_host(hh_ctx* ctx, int bits, const uint64_t* keys, int key_mode,
                 const uint8_t* bytes, const int64_t* offsets, int64_t n, uint64_t* out);

/*
 * Ragged-batch hash that allocates nothing.  The paper has no counterpart: it
 * serves callers that cannot allocate device memory for this library, because
 * another allocator owns their device memory (a framework's caching pool, or
 * a fixed budget that an out-of-band cudaMalloc would break) or because they
 * run on a latency-critical path where cudaMalloc's implicit device
 * synchronisation is not acceptable.
 *
 * Same hash and argument meaning as hh_hash{64,128,256}_batch (bits = 64,
 * 128 or 256; device pointers; asynchronous on `stream`), on the current
 * CUDA device, with no hh_ctx.  The length-sort scratch lives in a fixed
 * file-scope device array of about 4.03 MiB (room for
 * HH_NOALLOC_MAX_MESSAGES messages) that every GPU which loads the library
 * holds until the process exits; n > HH_NOALLOC_MAX_MESSAGES returns
 * HH_ERR_TOO_LARGE and enqueues nothing.  The call itself calls no
 * cudaMalloc, cudaFree or allocating routine.
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  All calls on a device share the one array, so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race
 * and give wrong results: serialise them.  Each call clears or rewrites
 * every part of the array it reads.  `device_error` is an optional device
 * int: when the device detects an error (decreasing offsets) the first such
 * hh_status code is written there; the call never clears it.  NULL
 * discards device errors.
 */
#define HH_NOALLOC_MAX_MESSAGES (1 << 20)
int hh_hash_batch_noalloc(int bits, const uint64_t* keys, int key_mode, const uint8_t* bytes,
                          const int64_t* offsets, int64_t n, uint64_t* out, int* device_error,
                          void* stream);

/*
 * SipTreeHash (Section 3), the paper's tree extension of SipHash, of a ragged
 * batch; 64-bit output.  Same keys, bytes, offsets, n and out conventions,
 * errors and asynchrony as hh_hash64_batch (and the same scratch limit);
 * `variant` is HH_SIPTREE (SipHash-2-4 lanes) or HH_SIPTREE13 (SipHash-1-3,
 * Section 5).  Section 3 fixes four interleaved SipHash lanes over 64-bit
 * words whose results are hashed again; the rest is read as follows: the
 * message is zero-padded to P = ceil(len / 32) vectors of 32 bytes; little-
 * endian word i goes to lane i mod 4; lane j is the standard SipHash of its
 * 8P bytes; the result is the standard SipHash of the four lane results
 * followed by len (five little-endian words); every SipHash is keyed with
 * key words 0 and 1 (words 2 and 3 are not used).
 */
enum hh_siptree_variant { HH_SIPTREE = 24, HH_SIPTREE13 = 13 };
int hh_siptree_batch(hh_ctx* ctx, int variant, const uint64_t* keys, int key_mode,
                     const uint8_t* bytes, const int64_t* offsets, int64_t n, uint64_t* out,
                     void* stream);

/*
 * Synchronise `stream`, then return and clear the context's device error
 * word: HH_OK, HH_ERR_BAD_OFFSETS, HH_ERR_BAD_KEY_INDEX, HH_ERR_BAD_CHUNK or
 * HH_ERR_TIMEOUT (the first one recorded).
 */
int hh_get_device_error(hh_ctx* ctx, void* stream);

/* Force one kernel family (enum hh_kernel) for later calls on ctx. */
int hh_set_kernel(hh_ctx* ctx, int kernel);

/* Batch regimes that have their own kernel shape. */
enum hh_regime {
  HH_REGIME_FIXED = 0,      /* hh_hash_fixed on 16-byte aligned lengths (TMA) */
  HH_REGIME_RAGGED = 1,     /* offsets-based calls (warp-tile kernel)         */
  HH_REGIME_BULK = 2        /* HH_KERNEL_STAGED_BULK                          */
};

/* Set a kernel shape for one regime: `window` bytes of every message staged
 * per pipeline step, `stages` pipeline buffers, and (fixed-length TMA kernel
 * only; 1 elsewhere) `messages_per_thread` interleaved messages per thread.
 * Supported (window, stages, messages_per_thread): HH_REGIME_FIXED
 * (128, 2..4, 1), (256, 2..3, 1), (128, 2..3, 2); HH_REGIME_RAGGED
 * (128, 2..4, 1), (256, 2..3, 1); HH_REGIME_BULK (128, 3..4, 1),
 * (256, 2..3, 1).  Others return HH_ERR_INVALID_ARG. */
int hh_set_staged_shape(hh_ctx* ctx, int regime, int window, int stages,
                        int messages_per_thread);

/*
 * Integer-issue microbenchmark (no counterpart in the paper; it measures the
 * ceiling the integer pipes put on Section 4.2's Update).  Each of `threads`
 * threads (a multiple of 32; of 256 when above 256) runs `updates` Updates
 * on register state with no memory traffic and writes one word to
 * out[thread] (device uint64 [threads]).  Variants 0..5 keep the whole
 * four-lane state in one thread and split the additions differently
 * between the ALU and FMA pipes; variants 6..11 are the same six splits for
 * one lane pair per thread (how messages of 128 KiB and more run).  The
 * variants of each group give identical output words.  Variant 12 keeps one
 * lane per thread (four threads per state; thread 4s + q holds lane q, its
 * packet word is its thread index, and it writes lane q of the output sum),
 * trading the ZipperMerge partner's upper half by warp shuffle.  With few
 * threads it measures the time of one Update chain rather than the pipes'
 * throughput.
 */
#define HH_UPDATE_VARIANTS 13
int hh_update_microbench(hh_ctx* ctx, int variant, int64_t updates, int64_t threads,
                         uint64_t* out, void* stream);

/*
 * Autotuner (no counterpart in the paper).  Times the candidate kernel
 * shapes on synthetic batches of at most `max_device_bytes` (>= 64 MiB; it
 * allocates that much plus small buffers, and frees them before returning)
 * and keeps, in ctx, the fastest per length regime: for fixed-length
 * batches per length class (<= 64, <= 256, <= 1024, <= 8192 bytes, larger)
 * the TMA kernel's window, pipeline depth and messages per thread; for
 * ragged batches the warp-tile kernel's window and depth; the message
 * length from which a message runs two threads per message (or never); and
 * up to how many such messages per SM each gets a warp of its own.
 * Synchronous; takes seconds.  Results are identical whatever is chosen.
 */
int hh_autotune(hh_ctx* ctx, int64_t max_device_bytes);

/*
 * Set one scalar of ctx's tuning table (the shapes are set with
 * hh_set_staged_shape).  Names and ranges:
 *   "huge_bucket"  0..4096: length-sort bucket from which messages run two
 *                  threads per message (4096: never; default 2176, 128 KiB);
 *   "solo_per_sm"  0..64: while at most this many such messages per SM are
 *                  in a launch, each gets a warp of its own (0: never;
 *                  default 4);
 *   "solo_shared"  0/1: whether those one-per-warp tiles are also used while
 *                  other launches with such messages are in flight (default
 *                  1);
 *   "fixed_pair"   0/1: whether fixed-length batches too small to give every
 *                  SM a tile run two threads per message (1, default) or
 *                  one.
 * HH_ERR_INVALID_ARG for another name or a value out of range.  Results
 * never depend on these settings.
 *
 * One more name sets a property of the context, not of the tuning table
 * (hh_tune_save does not write it):
 *   "wait_limit_ns" >= 0: how long a kernel waits for one asynchronous copy
 *                  before it gives up (default 2e9, 2 s; 0 tests the copy's
 *                  barrier once without blocking).  A kernel that gives up
 *                  records HH_ERR_TIMEOUT in the device error word, issues no
 *                  further copies, waits for the copies it issued (at most
 *                  0.2 s each) and writes zero hashes for the messages it
 *                  did not finish; messages it finished are hashed exactly.
 */
int hh_set_tune_param(hh_ctx* ctx, const char* name, int value);

/* Write ctx's tuning table as text (hh_init reads it back). */
int hh_tune_save(hh_ctx* ctx, const char* path);

/* The tuning table as text into buf (NUL-terminated), followed, after an
 * hh_autotune, by comment lines ('#') with each candidate's measured time;
 * HH_ERR_TOO_LARGE if buf_len is too small (8 KiB always suffices). */
int hh_tune_describe(hh_ctx* ctx, char* buf, int64_t buf_len);

/*
 * Streams: n messages that arrive in pieces (Section 4.5 adds the size
 * only at the end, so everything before the last piece is plain packets).
 * A stream's state is 16 uint64 words in caller-owned device memory,
 * states[m * 16 ..]: v0[0..3], v1[0..3], mul0[0..3], mul1[0..3].
 *
 * hh_stream_init: states[m] = Init(key of stream m) (key_mode as for
 * hh_hash*_batch; keys on the device).
 * hh_stream_update: appends piece m = bytes[offsets[m] .. offsets[m+1]) to
 * stream m.  Every piece must be a whole number of 32-byte packets (empty
 * is fine); a piece that is not sets HH_ERR_BAD_CHUNK in the device error
 * word and leaves that stream's state unchanged.
 * hh_stream_finish: appends the last piece m (any length), finalises and
 * writes stream m's `bits`-bit hash to out[m * bits / 64 ..]; the states
 * are read only.
 * The hash of a stream equals hh_hash*_batch of the concatenation of its
 * pieces.  All three are asynchronous on `stream`; the pointers are device
 * pointers; offsets are non-decreasing.  They run in the length-sorted
 * warp-tile kernels (HH_KERNEL_AUTO or HH_KERNEL_STAGED_UNSORTED; the naive
 * and bulk kernels return HH_ERR_INVALID_ARG).
 */
int hh_stream_init(hh_ctx* ctx, const uint64_t* keys, int key_mode, int64_t n,
                   uint64_t* states, void* stream);
int hh_stream_update(hh_ctx* ctx, uint64_t* states, const uint8_t* bytes, const int64_t* offsets,
                     int64_t n, void* stream);
int hh_stream_finish(hh_ctx* ctx, int bits, const uint64_t* states, const uint8_t* bytes,
                     const int64_t* offsets, int64_t n, uint64_t* out, void* stream);

/*
 * Counter-mode output (the paper names random-number generation as a use,
 * Sections 1 and 7): out[i] = HighwayHash-`bits`(key, m_i) for i < n, where
 * m_i is the 8-byte little-endian encoding of counter0 + i (mod 2^64).
 * `key`: device uint64[4]; `out`: device uint64[n * bits / 64].  Asynchronous
 * on `stream`; the same result as hashing those 8-byte messages with
 * hh_hash*_batch.
 */
int hh_prng_fill(hh_ctx* ctx, int bits, const uint64_t* key, uint64_t counter0, int64_t n,
                 uint64_t* out, void* stream);

/*
 * Statistical studies (the experiments of Sections 4.3 and 6; not part of
 * the hash).
 *
 * hh_stats_round_table: table[x] = the 64-bit hash, under `key` (HOST
 * uint64[4]) and with `rounds` (0..16) finalisation rounds instead of 4, of
 * the nbytes-byte (1..3) little-endian encoding of x, for every x below
 * 2^(8 nbytes).  `table`: device uint64[2^(8 nbytes)].
 *
 * hh_stats_toggle_counts: for a device table of 2^m words (m 1..30), adds to
 * counts[j * 64 + k] (device uint64[m * 64], zeroed by the caller) the
 * number of x < 2^m for which bit k of table[x] ^ table[x ^ 2^j] is set.
 * Every unordered pair is counted twice.
 *
 * hh_stats_avalanche: for t < iterations, the message is the first `size`
 * (1..32) bytes of the little-endian words splitmix64(seed, 4 + 4t + w),
 * w = 0..3, and the key is splitmix64(seed, 0..3), where splitmix64(s, c)
 * is output c of Vigna's splitmix64 started at state s.  Adds to
 * counts[b * 64 + k] (device uint64[8 size * 64], zeroed by the caller) how
 * many t flip output bit k of the 64-bit hash when input bit b flips.
 *
 * All three are asynchronous on `stream`.
 */
int hh_stats_round_table(hh_ctx* ctx, const uint64_t* key, int nbytes, int rounds,
                         uint64_t* table, void* stream);
int hh_stats_toggle_counts(hh_ctx* ctx, const uint64_t* table, int m, uint64_t* counts,
                           void* stream);
int hh_stats_avalanche(hh_ctx* ctx, int size, uint64_t seed, int64_t iterations,
                       uint64_t* counts, void* stream);

/* Number of kernel launches the last hash call on ctx enqueued. */
int hh_last_launch_count(hh_ctx* ctx);

/* A static, human-readable description of a status code. */
const char* hh_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HH_H */
