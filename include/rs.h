/*
 * rs -- LSD radix sort for NVIDIA GB300 (sm_103a).  C ABI.
 *
 * The method is the parallel LSD radix sort of Bozidar & Dobravec,
 * "Comparison of parallel sorting algorithms" (arXiv 1511.03404), Sec. 2.6:
 * keys are split into d digits of r bits; the sequence is sorted one digit
 * at a time from the least to the most significant digit, each time with a
 * stable counting sort (digit histogram, exclusive scan of the histogram,
 * stable scatter).  Sec. 1 and Sec. 3 ask for arbitrary lengths and for four
 * data types: 32-bit keys, 32-bit key-value pairs, 64-bit keys and 64-bit
 * key-value pairs.
 *
 * Conventions shared by every entry point below:
 *   - Order: ascending unsigned order of the key bits [begin_bit, end_bit).
 *     Bits outside that range are ignored (but kept).  The sort is stable:
 *     elements with equal key bits keep their input order.
 *   - Pairs are structure-of-arrays: keys[i] and vals[i] belong together.
 *     Values have the width of the keys (u32 with u32 keys, u64 with u64).
 *   - Device pointers.  keys/vals/keys_alt/vals_alt, the workspace and every
 *     other buffer named "d_" or "device" are device memory of the current
 *     CUDA device, owned by the caller; the library never allocates, frees
 *     or retains them past the call.  Keys and values must be aligned to
 *     their element size; the workspace to 256 bytes.
 *   - Double buffering.  keys_alt/vals_alt are caller-owned buffers of the
 *     same size as keys/vals.  On return *result_in_alt tells where the
 *     sorted sequence will be: 0 = keys/vals, 1 = keys_alt/vals_alt.  The
 *     other pair of buffers holds unspecified data afterwards.  The input is
 *     not preserved.
 *   - Asynchrony.  Sorts are enqueued on `stream` (a cudaStream_t; NULL is
 *     the legacy default stream) and return before the work completes.
 *     The call itself never synchronizes.  All kernels of one call go on
 *     that one stream, so a call can be captured into a CUDA graph.
 *   - Errors.  Every call returns an rs_status.  Argument errors are found on
 *     the host before anything is enqueued (RS_ERR_INVALID,
 *     RS_ERR_WORKSPACE).  Launch failures give RS_ERR_CUDA.  Errors that can
 *     only be seen on the device (a bounded wait that ran out, an index
 *     check that failed) are recorded in a status word inside the workspace;
 *     read it with rs_workspace_status() after the stream's work is done.
 *     Every sort given a workspace of at least 256 bytes resets that status
 *     word, even on paths that need no other workspace.
 *     The library never aborts, traps or hangs: every device-side wait is
 *     bounded in time.
 *   - Limits: n <= RS_MAX_N.  0 <= begin_bit <= end_bit <= key bits.
 */
#ifndef RS_H_
#define RS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* rs_stream_t;

/* Largest supported number of elements in one array or one segment.  The
 * look-back status words carry a 30-bit running count. */
#define RS_MAX_N ((size_t)((1u << 30) - 1u))

typedef enum rs_status {
  RS_OK = 0,
  RS_ERR_INVALID = 1,   /* bad argument: null pointer, misalignment, size or bit range */
  RS_ERR_NOMEM = 2,     /* an allocation the call needed (server pool) failed */
  RS_ERR_CUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  RS_ERR_TIMEOUT = 4,   /* a bounded device-side wait (decoupled look-back) ran out */
  RS_ERR_BUSY = 5,      /* server: request not admitted now (queue full / over budget) */
  RS_ERR_WORKSPACE = 6, /* workspace missing, too small or misaligned */
  RS_ERR_DEVICE = 7,    /* a device-side index check failed; output not valid */
  RS_ERR_CANCELLED = 8, /* server: request cancelled before it ran */
  RS_ERR_NOT_FOUND = 9  /* server: unknown handle */
} rs_status;

/* Human-readable name of a status code (static string). */
const char* rs_status_string(rs_status s);

/* Library version as "major.minor.patch" (static string). */
const char* rs_version(void);

/* How the key bits are read (rs_config.key_kind). */
typedef enum rs_key_kind {
  RS_KEY_UNSIGNED = 0, /* unsigned integers (the paper's keys, Sec. 3) */
  RS_KEY_SIGNED = 1,   /* two's-complement signed integers of key_bytes */
  RS_KEY_FLOAT = 2     /* IEEE-754 binary32 (key_bytes 4) or binary64 (key_bytes 8) */
} rs_key_kind;

/*
 * Tuning parameters and key order.  radix_bits is the digit width r of
 * Sec. 2.6; the sorted result does not depend on it.  variant selects one of
 * the compiled tile shapes (threads per CTA x keys per thread), see
 * rs_variant_info().  A zero / negative tuning field means "let the library
 * choose" (the tuned table).  A zero-initialised struct sorts unsigned keys
 * in ascending order.
 *
 * key_kind and descending extend the paper's unsigned LSD sort (its digit
 * decomposition is defined on unsigned integers) by an order-preserving bit
 * transform T applied to each key before its digits are taken, and undone
 * on the way out; the keys returned are the caller's own bit patterns.
 *   signed:  T flips the sign bit.
 *   float:   T flips every bit of a negative value and the sign bit of a
 *            non-negative one, giving the total order
 *            -NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN
 *            (-0.0 sorts before +0.0; NaNs sort by sign and payload).
 *   descending: T additionally inverts every bit.
 * The sort stays stable in every mode: equal keys (equal bit patterns) keep
 * their input order, also when descending.  begin_bit / end_bit select bits
 * of the transformed key.
 */
typedef struct rs_config {
  int radix_bits; /* 0: library choice; else one of the compiled widths */
  int variant;    /* -1: library choice; else an index from rs_variant_info */
  int key_kind;   /* rs_key_kind; any other value is RS_ERR_INVALID */
  int descending; /* 0: ascending, 1: descending; any other value is RS_ERR_INVALID */
} rs_config;

/* Number of compiled tile variants for (key_bytes, val_bytes); val_bytes 0 = keys only. */
int rs_num_variants(int key_bytes, int val_bytes);

/*
 * Describe variant `index` of (key_bytes, val_bytes): digit width, threads
 * per CTA, keys per thread, and kind (0 = multi-CTA onesweep with one CTA per
 * tile, 1 = one CTA sorting the whole array in shared memory, 2 = onesweep on
 * resident CTAs that each take tile after tile, 3 = the whole sort in one
 * cooperative launch with grid barriers between the passes, 4 = one
 * thread-block cluster sorting the whole array in its distributed shared
 * memory); max_n bounds the array size.
 */
rs_status rs_variant_info(int key_bytes, int val_bytes, int index, int* radix_bits,
                          int* threads, int* items_per_thread, int* kind, size_t* max_n);

/*
 * Tuned variant table (written by the package's autotuner): for sorts of
 * (key_bytes, val_bytes) with no explicit configuration, n <= n_max uses
 * `variant` (the entry with the smallest n_max >= n wins; n above every
 * entry falls back to the built-in choice).  Setting an existing n_max
 * replaces its variant.  RS_ERR_INVALID for an unknown type or variant.
 * Workspace sizes follow the table: query rs_workspace_bytes after changing
 * it.  rs_tune_clear drops every entry.  The library starts with the
 * package's tuned table as it was when the library was built (tuned.json),
 * unless the environment sets RS_NO_TUNED_TABLE when the table is first used.
 */
rs_status rs_tune_set(int key_bytes, int val_bytes, size_t n_max, int variant);
rs_status rs_tune_clear(void);

/*
 * Workspace bytes a sort of n elements over [begin_bit, end_bit) needs with
 * configuration cfg (NULL = library choice).  The sort entry points with the
 * same arguments accept any workspace at least this large.
 */
rs_status rs_workspace_bytes(int key_bytes, int val_bytes, size_t n, int begin_bit, int end_bit,
                             const rs_config* cfg, size_t* bytes);

/*
 * Sort 32-bit keys (Sec. 2.6 over 32-bit keys, Sec. 3).
 *   keys      [n] u32, device: input; may receive the output (see result_in_alt)
 *   keys_alt  [n] u32, device: the second buffer of the double buffer
 *   ws        device workspace of at least rs_workspace_bytes(4, 0, ...) bytes
 *   result_in_alt  host int, set before return: 1 if the sorted keys end in keys_alt
 */
rs_status rs_sort_keys_u32(uint32_t* keys, uint32_t* keys_alt, size_t n, int begin_bit,
                           int end_bit, void* ws, size_t ws_bytes, rs_stream_t stream,
                           int* result_in_alt);

/* Sort 64-bit keys (Sec. 2.6 over 64-bit keys, Sec. 3).  As rs_sort_keys_u32. */
rs_status rs_sort_keys_u64(uint64_t* keys, uint64_t* keys_alt, size_t n, int begin_bit,
                           int end_bit, void* ws, size_t ws_bytes, rs_stream_t stream,
                           int* result_in_alt);

/*
 * Sort 32-bit key-value pairs by key (Sec. 2.6, Sec. 3), stable.
 *   vals / vals_alt  [n] u32 device buffers that travel with keys / keys_alt.
 */
rs_status rs_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                            uint32_t* vals_alt, size_t n, int begin_bit, int end_bit, void* ws,
                            size_t ws_bytes, rs_stream_t stream, int* result_in_alt);

/* Sort 64-bit key-value pairs by key (Sec. 2.6, Sec. 3), stable. */
rs_status rs_sort_pairs_u64(uint64_t* keys, uint64_t* vals, uint64_t* keys_alt,
                            uint64_t* vals_alt, size_t n, int begin_bit, int end_bit, void* ws,
                            size_t ws_bytes, rs_stream_t stream, int* result_in_alt);

/* Largest n that rs_sort_keys_u32_noalloc accepts, and the size of the
 * fixed device array that serves as its workspace. */
#define RS_NOALLOC_MAX_N ((size_t)1 << 23)
#define RS_NOALLOC_SCRATCH_BYTES ((size_t)9 << 20)

/*
 * rs_sort_keys_u32 without a workspace argument and without allocating.
 * The paper has no counterpart: this entry exists for callers that may not
 * call cudaMalloc (or any allocator) at the point where they sort -- code
 * running inside a framework that owns every device byte through its own
 * pool, real-time or callback contexts where an allocation could block or
 * synchronize the device, and systems whose memory must all be reserved at
 * start-up.  The scratch it needs (RS_NOALLOC_SCRATCH_BYTES, 9 MiB) is a
 * fixed array of device memory inside this library, present on every GPU
 * that loads the library until the process exits.  The tile shape is the
 * library's usual choice when its workspace fits the array, else the compiled
 * shape with the smallest workspace; the sorted result is the same.
 *   keys, keys_alt, n, begin_bit, end_bit, stream, result_in_alt: as for
 *   rs_sort_keys_u32; n must not exceed RS_NOALLOC_MAX_N (else RS_ERR_INVALID,
 *   nothing enqueued).
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * All calls on a device share the one array and each call leaves its
 * contents behind (the next call clears what must start at zero): calls whose
 * work may overlap on the GPU, for example on two streams, race and must be
 * serialized by the caller.  The device address of the array is cached per
 * device for the life of the CUDA context it was looked up in: do not call
 * this entry point on a device after cudaDeviceReset of that device.
 */
rs_status rs_sort_keys_u32_noalloc(uint32_t* keys, uint32_t* keys_alt, size_t n, int begin_bit,
                                   int end_bit, rs_stream_t stream, int* result_in_alt);

/*
 * Device-side status of the last rs_sort_keys_u32_noalloc call on the current
 * device: synchronizes `stream` (the stream that call used), then reads the
 * status word in the library's array.  RS_OK, RS_ERR_TIMEOUT (a bounded wait
 * ran out) or RS_ERR_DEVICE (an index check failed; the output is not valid);
 * *info (may be NULL) receives the tile or pass that reported it.  Allocates
 * nothing.
 */
rs_status rs_sort_keys_u32_noalloc_status(rs_stream_t stream, uint32_t* info);

/*
 * Generic form of the four sorts above with an explicit configuration
 * (cfg may be NULL: unsigned ascending, library-chosen tuning).  key_bytes is
 * 4 or 8; val_bytes is 0 (keys only) or equal to key_bytes.  vals / vals_alt
 * must be NULL when val_bytes is 0.  cfg->key_kind and cfg->descending
 * choose the key order (see rs_config); a bad value is RS_ERR_INVALID with
 * nothing enqueued.
 */
rs_status rs_sort(int key_bytes, int val_bytes, void* keys, void* vals, void* keys_alt,
                  void* vals_alt, size_t n, int begin_bit, int end_bit, const rs_config* cfg,
                  void* ws, size_t ws_bytes, rs_stream_t stream, int* result_in_alt);

/*
 * End-to-end form of rs_sort for data in host memory: copies the caller's
 * host arrays into the device buffers, sorts them (Sec. 2.6, as rs_sort) and
 * copies the sorted arrays back, all enqueued on `stream` in that order.
 *   h_keys, h_vals          [n] host input (h_vals NULL when val_bytes is 0);
 *                           read by the copy engine after the call returns
 *   h_out_keys, h_out_vals  [n] host output; written when the stream's work
 *                           is done (may alias the input arrays)
 *   keys, vals, keys_alt, vals_alt, ws: device buffers as for rs_sort (the
 *                           caller owns them; the result is also left in the
 *                           pair that *result_in_alt names)
 * Asynchronous: the host arrays must stay valid until the stream has passed
 * this call's work (cudaStreamSynchronize, an event).  With page-locked host
 * memory (cudaHostAlloc / cudaHostRegister) the copies run on the copy
 * engines and overlap kernels of other streams, so calls on several streams,
 * each with its own buffers, form a copy-in / sort / copy-out pipeline;
 * pageable memory makes the copies synchronous.  Argument errors are found
 * before anything is enqueued (RS_ERR_INVALID, RS_ERR_WORKSPACE);
 * device-side status as for rs_sort (rs_workspace_status).
 */
rs_status rs_sort_host(int key_bytes, int val_bytes, const void* h_keys, const void* h_vals,
                       void* h_out_keys, void* h_out_vals, size_t n, int begin_bit, int end_bit,
                       const rs_config* cfg, void* keys, void* vals, void* keys_alt,
                       void* vals_alt, void* ws, size_t ws_bytes, rs_stream_t stream,
                       int* result_in_alt);

/*
 * What the last sort that used workspace `ws` did, read back after `stream`
 * is done: the digit passes that moved the data and those skipped because
 * one digit value held every key (Sec. 2.6's counting sort of that digit is
 * then the identity), the device time of each kernel phase, and the
 * algorithmic bytes.  Recorded by rs_sort, the four typed sorts,
 * rs_sort_host and rs_sort_keys_u32_noalloc (whose array has no public
 * address: its record is not readable).  A segmented sort's workspace gives
 * form 0; a workspace last used by the sample-sort, merge-sort or server
 * entry points holds no record.  Times come from the GPU's global timer and
 * include no host overhead.
 */
typedef struct rs_sort_stats {
  int status;            /* device-side status, as rs_workspace_status returns it */
  uint32_t info;         /* tile or pass that reported a device-side error */
  int form;              /* 0: no record; 1: digit histograms + one launch per pass;
                            2: the whole sort in one cooperative launch; 3: one CTA
                            (or cluster) holding the array in shared memory */
  int key_bytes, val_bytes, passes; /* passes = ceil((end_bit - begin_bit) / radix_bits) */
  uint64_t n;
  uint32_t moved_mask;   /* bit p: pass p read and wrote the data */
  uint32_t skipped_mask; /* bit p: pass p was skipped (forms 1 and 2) */
  double upsweep_ms;     /* forms 1, 2: start until every digit histogram and scan is
                            done; form 3: the whole sort */
  double pass_ms[16];    /* forms 1, 2: per moving pass, its first tile taken until its
                            last CTA finished; 0 for skipped passes */
  double total_ms;       /* first kernel's start until the last recorded time */
  double bytes;          /* algorithmic bytes: n K for the histograms plus
                            2 n (K + V) per moving pass (form 3: 2 n (K + V)) */
} rs_sort_stats;

/* Synchronizes `stream`, then fills *out.  RS_ERR_INVALID for out NULL;
 * RS_ERR_CUDA if the synchronization or the read failed.  A workspace that
 * holds no record (a segmented sort's, one never used) gives form 0. */
rs_status rs_workspace_stats(const void* ws, rs_stream_t stream, rs_sort_stats* out);

/*
 * Sample sort (Sec. 2.7), the regular-sampling variant after Dehne et al.,
 * as an MSD partition front end for 32-bit key-value pairs.
 *   1. The input is cut into blocks of 4096 pairs and every block is sorted
 *      stably, in place in keys / vals (they are overwritten).
 *   2. From each sorted block of L pairs, `samples` keys are taken at
 *      positions floor(j * L / samples), j = 0 .. samples - 1.
 *   3. The samples are sorted; splitter q (q = 0 .. buckets - 2) is the
 *      sorted sample at rank floor((q + 1) * M / buckets), M samples in all.
 *   4. A pair with key x belongs to bucket q = the number of splitters < x
 *      (equal keys always share a bucket).
 *   5. keys_out / vals_out receive the buckets in order; bucket q holds,
 *      block after block, each block's run of bucket-q pairs, so every key
 *      of bucket q lies in (splitter[q-1], splitter[q]] and pairs of equal
 *      keys keep their input order.
 *   keys, vals          [n] u32 device; overwritten (block-sorted)
 *   keys_out, vals_out  [n] u32 device, distinct from keys / vals
 *   samples             1 .. 4096 samples per block
 *   buckets             2 .. 4096 buckets (nblocks * buckets < 2^32)
 *   d_bucket_offsets    [buckets + 1] u64 device: bucket q is
 *                       [off[q], off[q+1]) of keys_out
 *   d_splitters         [buckets - 1] u32 device, or NULL
 *   ws                  device workspace of rs_sample_workspace_bytes() bytes,
 *                       256-byte aligned
 * Asynchronous on `stream`.  Bad sizes, pointers or alignment:
 * RS_ERR_INVALID with nothing enqueued; workspace too small:
 * RS_ERR_WORKSPACE.  Device-side status words of the sorts it runs are
 * read with rs_workspace_status on the segmented part of ws (not needed in
 * normal use).
 */
rs_status rs_sample_workspace_bytes(size_t n, int samples, int buckets, size_t* bytes);
rs_status rs_sample_partition_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_out,
                                        uint32_t* vals_out, size_t n, int samples, int buckets,
                                        uint64_t* d_bucket_offsets, uint32_t* d_splitters,
                                        void* ws, size_t ws_bytes, rs_stream_t stream);

/*
 * Sample sort of 32-bit pairs: the partition above, then every bucket sorted
 * by the LSD radix sort (one batched segmented sort, Sec. 2.7's "alternative
 * sort").  The result equals rs_sort_pairs_u32's (stable, ascending);
 * *result_in_alt = 1 when it is in keys_out / vals_out (always, for n > 0),
 * 0 when in keys / vals.  Arguments as for rs_sample_partition_pairs_u32.
 */
rs_status rs_sample_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_out,
                                   uint32_t* vals_out, size_t n, int samples, int buckets,
                                   uint64_t* d_bucket_offsets, void* ws, size_t ws_bytes,
                                   rs_stream_t stream, int* result_in_alt);

/*
 * Merge sort (Sec. 2.4; the parallel merge sort of Satish et al.): a stable
 * comparison sort, ascending, for keys the radix passes do not take as well
 * as for 32- and 64-bit keys.
 *   key_bytes 4 (u32), 8 (u64) or 16: a 128-bit unsigned key stored as two
 *             little-endian u64 words (value = word0 + 2^64 * word1), array
 *             16-byte aligned
 *   val_bytes 0, or the key width for 4 / 8-byte keys, or 8 for 16-byte keys
 *   keys, vals, keys_alt, vals_alt  [n] device arrays (double buffer); the
 *             result ends in keys / vals (*result_in_alt = 0) or in the
 *             alternates (1): the parity of the number of merge passes,
 *             ceil(log2(ceil(n / 4096)))
 *   ws        device workspace of rs_merge_workspace_bytes() bytes, 256-byte
 *             aligned (the merge-path split of every output tile)
 * Tiles of 4096 elements are sorted inside one CTA each, then runs are merged
 * pairwise, each CTA producing one tile of the output from the two input
 * ranges a merge-path search delimits.  Equal keys keep their input order.
 * Asynchronous on `stream`.  Bad types, sizes, pointers or alignment:
 * RS_ERR_INVALID; workspace too small: RS_ERR_WORKSPACE; both with nothing
 * enqueued.
 */
rs_status rs_merge_workspace_bytes(int key_bytes, int val_bytes, size_t n, size_t* bytes);
rs_status rs_merge_sort(int key_bytes, int val_bytes, void* keys, void* vals, void* keys_alt,
                        void* vals_alt, size_t n, void* ws, size_t ws_bytes, rs_stream_t stream,
                        int* result_in_alt);

/*
 * Digit histograms and their exclusive scans, the first two steps of each
 * counting sort of Sec. 2.6, for every digit pass at once.
 *   keys         [n] device keys of key_bytes (4 or 8); not modified
 *   d_counts     [passes * 2^radix_bits] u32 device: counts[p][v] = number of
 *                keys whose digit p equals v
 *   d_offsets    [passes * 2^radix_bits] u32 device: offsets[p][v] =
 *                sum of counts[p][u] over u < v
 *   d_exec_mask  [1] u32 device: bit p set when pass p moves data (no single
 *                digit value holds all n keys), after the parity rule that
 *                keeps the number of moving passes congruent to `passes` mod 2
 * passes = ceil((end_bit - begin_bit) / radix_bits).  Uses workspace like a
 * sort of the same keys.
 */
rs_status rs_digit_counts(int key_bytes, const void* keys, size_t n, int begin_bit, int end_bit,
                          int radix_bits, uint32_t* d_counts, uint32_t* d_offsets,
                          uint32_t* d_exec_mask, void* ws, size_t ws_bytes, rs_stream_t stream);

/*
 * Wait for `stream` and report the device-side status of the last call that
 * used workspace `ws`: RS_OK, RS_ERR_TIMEOUT or RS_ERR_DEVICE (RS_ERR_CUDA if
 * the synchronization itself failed).  *info (may be NULL) receives the tile
 * or pass the device reported.
 */
rs_status rs_workspace_status(const void* ws, rs_stream_t stream, uint32_t* info);

/*
 * Batched segmented sort of 32-bit key-value pairs: the sort of Sec. 2.6
 * applied independently to every segment of one array, in a fixed sequence of
 * launches whatever the segments: a one-CTA planning launch, one kernel for the
 * short segments, one for the long segments' histograms and one persistent
 * kernel for all their passes.
 *   keys, vals, keys_alt, vals_alt  [n] u32 device buffers as for rs_sort_pairs_u32
 *   d_offsets  [n_seg + 1] u64 device: segment s is [d_offsets[s], d_offsets[s+1]);
 *              d_offsets[0] = 0, non-decreasing, d_offsets[n_seg] = n, and no
 *              segment longer than RS_MAX_N.  Offsets that break these rules are
 *              reported by rs_workspace_status() as RS_ERR_INVALID and no
 *              element is written.
 * Every segment is sorted over [begin_bit, end_bit), stable.  *result_in_alt
 * (host) names the buffer pair that holds every sorted segment; it depends
 * only on the bit range: 1 when ceil((end_bit - begin_bit) / 8) is odd.
 * ws: at least rs_segmented_workspace_bytes(n, n_seg, ...) bytes, 256-aligned.
 * The host reads nothing from the device: the plan is made on the GPU.
 */
rs_status rs_segmented_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                                  uint32_t* vals_alt, size_t n, const uint64_t* d_offsets,
                                  size_t n_seg, int begin_bit, int end_bit, void* ws,
                                  size_t ws_bytes, rs_stream_t stream, int* result_in_alt);

/* Workspace bytes rs_segmented_sort_pairs needs for n elements in n_seg segments. */
rs_status rs_segmented_workspace_bytes(size_t n, size_t n_seg, int begin_bit, int end_bit,
                                       size_t* bytes);

/*
 * The batched segmented sort for any of the four data types of Sec. 3:
 * key_bytes 4 or 8, val_bytes 0 (keys only) or equal to key_bytes; vals and
 * vals_alt must be NULL when val_bytes is 0.  Everything else as for
 * rs_segmented_sort_pairs (offsets, bit range up to 8 * key_bytes, result
 * buffer by the pass count's parity, status through rs_workspace_status),
 * with rs_segmented_workspace_bytes_typed for the workspace.  Segments of
 * up to 4096 elements (2048 for 64-bit keys) are sorted whole by one CTA.
 */
rs_status rs_segmented_sort(int key_bytes, int val_bytes, void* keys, void* vals, void* keys_alt,
                            void* vals_alt, size_t n, const uint64_t* d_offsets, size_t n_seg,
                            int begin_bit, int end_bit, void* ws, size_t ws_bytes,
                            rs_stream_t stream, int* result_in_alt);
rs_status rs_segmented_workspace_bytes_typed(int key_bytes, int val_bytes, size_t n, size_t n_seg,
                                             int begin_bit, int end_bit, size_t* bytes);

/* ---- sort server: continuous batching of requests on one GPU ---------- */

/*
 * A server owns one resident device-memory pool of `budget_bytes` (allocated
 * once by rs_server_create) and `streams` CUDA streams on the device that is
 * current at creation.  A scheduler thread admits queued requests, oldest
 * first, whenever the request's device footprint fits the free part of the
 * pool and a stream is free; a request that does not fit yet does not block
 * younger ones that do.  Requests of at most batch_max_n elements (2^14 by
 * default, see rs_server_config) that wait together and share key and value
 * widths and bit range are packed into one batched segmented sort, which
 * takes a free stream before any single request does; every other request
 * (and a short one waiting alone) runs as its own sort, large ones (large_n
 * elements and up) at most max_large at a time.  Each admitted unit runs
 * copy-in, sort, copy-out on its stream, so units overlap on the device;
 * with shared copy queues (an option) the copies in of all units of a size
 * class (large or not) go through one FIFO copy stream and their copies out
 * through another, ordered against the unit's sort by events.
 * The sorted result of a request does not depend on what it was batched or
 * overlapped with.
 */
typedef struct rs_server rs_server;
typedef uint64_t rs_handle;

typedef struct rs_request {
  int key_bytes;          /* 4 or 8 */
  int val_bytes;          /* 0 or key_bytes */
  size_t n;               /* elements, <= RS_MAX_N */
  int begin_bit, end_bit; /* key bits to sort by */
  const void* h_keys;     /* [n] host input keys (pinned memory lets copies overlap) */
  const void* h_vals;     /* [n] host input values, or NULL when val_bytes is 0 */
  void* h_out_keys;       /* [n] host output: the sorted keys */
  void* h_out_vals;       /* [n] host output: the values in key order, or NULL */
} rs_request;
/* The host buffers must stay valid and untouched until rs_poll reports the
 * request done.  Input and output may be the same buffers. */

typedef struct rs_server_stats_t {
  uint64_t completed, failed, keys;   /* requests done (ok / with an error), keys sorted */
  uint64_t batches, batched_requests; /* segmented launches and the requests they carried */
  uint64_t queued, max_queued;        /* requests waiting now / at most */
  size_t pool_peak_bytes, pool_used_bytes;
  double p50_ms, p99_ms, max_ms;      /* submit -> done latency of completed requests */
  double wall_s;                      /* first submit -> last completion */
  double gkeys_per_s;                 /* keys / wall_s / 1e9 */
  double wait_p50_ms, wait_p99_ms;    /* submit -> admission (queueing) */
  double service_p50_ms, service_p99_ms; /* admission -> done (copies, sort, callback) */
} rs_server_stats_t;

/* One completed request, as recorded by the server: times in seconds since
 * the first submission after creation or the last rs_server_reset_stats. */
typedef struct rs_trace_record {
  double submit_s, admit_s, done_s; /* submitted, admitted to a stream, completion callback */
  uint64_t n;                       /* elements */
  int key_bytes, val_bytes;
  int stream;                       /* server stream it ran on */
  int batched;                      /* 1: shared a batched segmented launch */
} rs_trace_record;

/* Create a server: budget_bytes >= 1 MiB of device memory, 1..64 streams.
 * RS_ERR_NOMEM if the pool cannot be allocated. */
rs_status rs_server_create(size_t budget_bytes, int streams, rs_server** out);

/* Scheduling policy of a server (rs_server_get_config / rs_server_set_config).
 * A new setting applies to admissions after the call; running units keep
 * theirs.  Defaults in brackets. */
typedef struct rs_server_config {
  size_t batch_max_n;    /* requests of 2..batch_max_n elements are batched [2^14] */
  size_t max_batch_keys; /* elements per batched launch at most, >= batch_max_n [2^22] */
  size_t large_n;        /* requests of at least large_n elements are "large" [2^21] */
  int max_large;         /* large units admitted at once, oldest first, 1..64 [3] */
  int large_low_priority; /* 1: large units run on low-priority streams, so that the
                             kernels of short requests are scheduled ahead of them [1] */
  int shared_copy_queues; /* 1: copies through one FIFO copy stream per direction and
                             size class; 0: on each unit's own stream [0] */
} rs_server_config;

/* RS_ERR_INVALID for a NULL argument or a field out of range
 * (batch_max_n > max_batch_keys, max_batch_keys > RS_MAX_N, large_n = 0,
 * max_large outside 1..64, large_low_priority or shared_copy_queues not 0
 * or 1). */
rs_status rs_server_get_config(rs_server* server, rs_server_config* out);
rs_status rs_server_set_config(rs_server* server, const rs_server_config* cfg);

/* Stop the scheduler after the requests already on the GPU finish; queued
 * requests end as RS_ERR_CANCELLED.  Frees the pool and the streams. */
rs_status rs_server_destroy(rs_server* server);

/* Queue a request without blocking.  RS_ERR_INVALID for a malformed request
 * or one whose footprint exceeds the whole budget; RS_ERR_BUSY when the server
 * is stopping or the queue is full. */
rs_status rs_submit(rs_server* server, const rs_request* req, rs_handle* out);

/* Non-blocking completion check.  *done = 0: still queued or running (returns
 * RS_OK).  *done = 1: finished; the return value is the request's status
 * (RS_OK, RS_ERR_CANCELLED, RS_ERR_TIMEOUT, ...) and the handle is retired
 * (a later poll returns RS_ERR_NOT_FOUND). */
rs_status rs_poll(rs_server* server, rs_handle handle, int* done);

/* Cancel a request that has not started (RS_ERR_BUSY once it is on the GPU). */
rs_status rs_cancel(rs_server* server, rs_handle handle);

/* Completion queue: move up to `cap` handles of requests that finished (done,
 * failed or cancelled) since the last call, oldest first, into out[0 .. *count).
 * rs_poll on such a handle then reports its status without waiting.  One call
 * replaces polling every pending handle, so a client with many requests in
 * flight does not contend with the scheduler for the server's lock.  The
 * queue holds at most 2^20 handles; older ones are dropped (rs_poll still
 * finds them). */
rs_status rs_server_completed(rs_server* server, rs_handle* out, size_t cap, size_t* count);

/* Latency percentiles, throughput and pool use since creation or the last reset. */
rs_status rs_server_stats(rs_server* server, rs_server_stats_t* out);
rs_status rs_server_reset_stats(rs_server* server);

/*
 * Copy the records of completed requests (in completion order) into
 * out[0 .. min(cap, total)); *total receives how many there are.  out may be
 * NULL with cap 0 to ask for the count.  The server keeps every record until
 * rs_server_reset_stats.
 */
rs_status rs_server_trace(rs_server* server, rs_trace_record* out, size_t cap, size_t* total);

/* ---- per-kernel timing (CUDA events recorded on the sort's stream) ---- */

/* Kinds of kernels the library launches. */
typedef enum rs_kernel_kind {
  RS_KERNEL_UPSWEEP = 0, /* digit histograms of all passes + scan */
  RS_KERNEL_ONESWEEP = 1, /* one digit pass: rank, look-back, stable scatter */
  RS_KERNEL_SMALL = 2,   /* whole array sorted by one CTA in shared memory */
  RS_KERNEL_SEGMENTED = 3, /* batched segments */
  RS_KERNEL_MERGE = 4,   /* merge sort: tile sort or one merge pass */
  RS_KERNEL_SAMPLE = 5,  /* sample-sort partition: bucket counts or the run copy */
  RS_KERNEL_KINDS = 6
} rs_kernel_kind;

/*
 * Start recording: every later kernel launch of this library on this host
 * thread is bracketed by CUDA events (up to `capacity` launches).  Calling
 * it again discards earlier records.
 */
rs_status rs_profile_begin(int capacity);

/*
 * Stop recording, wait for the recorded events and return, per kernel kind,
 * the number of launches, their summed duration in milliseconds and their
 * summed algorithmic bytes (reads + writes the method needs: for a onesweep
 * pass 2 n (key bytes + value bytes), for the upsweep n key bytes, for a
 * merge pass 2 n (key bytes + value bytes), for the sample-sort bucket
 * counts n key bytes and for its run copy 2 n (key bytes + value bytes)).  Arrays
 * have RS_KERNEL_KINDS entries; any may be NULL.
 */
rs_status rs_profile_end(int* launches, double* ms, double* bytes);

/* ---- fault injection for tests (host-set, off by default) ---- */

typedef enum rs_debug_knob {
  RS_DEBUG_TIMEOUT_NS = 0,        /* look-back wait limit in ns (default 1e9) */
  RS_DEBUG_DROP_PUBLISH_TILE = 1, /* tile that never publishes its look-back status; -1 off */
  RS_DEBUG_DROP_PUBLISH_PASS = 2, /* pass in which that tile stays silent */
  RS_DEBUG_TRACE_PTR = 3,         /* device u64 buffer [tiles][16] for onesweep phase data; 0 off */
  RS_DEBUG_TRACE_TILES = 4,       /* number of tiles the trace buffer holds */
  RS_DEBUG_TRACE_PASS = 5,        /* the digit pass whose tiles are traced */
  RS_DEBUG_LB_SMALL = 6,          /* look-back windows of 8 status words instead of 32 */
  RS_DEBUG_BAD_INDEX_TILE = 7     /* debug build only (else RS_ERR_INVALID): this tile of
                                     digit pass 0 of a multi-launch sort computes scatter
                                     indices past the array, so that the bounds checks of
                                     rs_debug_status must catch and drop them; -1 off */
} rs_debug_knob;

/* Set a knob for later calls from any thread; returns RS_ERR_INVALID for an unknown knob. */
rs_status rs_debug_set(rs_debug_knob knob, long long value);

/*
 * Bounds checks of a debug build.  The library built with RS_DEBUG defined
 * (the package's build step writes it as _build/librs_debug.so beside
 * librs.so) checks the index of every global store of its kernels against
 * the length of the array it writes; an index out of range is recorded (the
 * first one per compiled unit: a store-site number and the index) and the
 * store is dropped; nothing traps.  This call synchronizes the current
 * device, then reads and clears those records: RS_ERR_DEVICE if a check
 * failed since the last call (*site, *index: the first one found), else
 * RS_OK.  *debug_build (may be NULL) is 1 in a debug build; in a release
 * build nothing is checked and the call returns RS_OK without touching the
 * device.  Not part of any sort's status: use it in tests.
 */
rs_status rs_debug_status(int* debug_build, uint32_t* site, uint64_t* index);

#ifdef __cplusplus
}
#endif

#endif /* RS_H_ */
