/*
 * Oracle for the LSD radix sort -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, __graft_entry__.smoke() and the benchmark's CPU-baseline
 * leg may load this file's library.  The product path (the CUDA library under
 * paper_1511_03404_gb300/) never calls it, and the two share no code.
 *
 * What it computes (arXiv 1511.03404, Sec. 2.6): the keys are split into
 * d digits of r bits each; the sequence is then sorted by one digit at a time,
 * least significant digit first, with a stable counting sort, so that
 * elements whose current digits are equal keep the order the previous digit
 * left them in.  One counting-sort step is
 *     1. count[v]  = number of elements whose digit equals v,
 *     2. start[v]  = sum of count[u] over u < v   (exclusive prefix),
 *     3. for i = 0, 1, ..., n-1 in input order:
 *            out[start[digit(i)]++] = element i.
 * After the last digit the sequence is in ascending unsigned order of the key
 * bits [begin_bit, end_bit), and elements with equal key bits are in their
 * input order (the sort is stable).  Values, when present, travel with their
 * keys.  Every digit is processed: the oracle never skips a digit.
 *
 * The digit of pass p is bits [begin_bit + p*r, min(begin_bit + (p+1)*r,
 * end_bit)) of the key; the number of passes is ceil((end_bit-begin_bit)/r).
 *
 * Plain C, single thread, no blocking or fusion.  Each step above is a
 * separate loop.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

/* Number of digit passes for the key bits [begin_bit, end_bit) at r bits. */
int oracle_num_passes(int key_bits, int begin_bit, int end_bit, int r) {
  if (r < 1 || r > 16 || begin_bit < 0 || end_bit > key_bits || begin_bit > end_bit)
    return -1;
  return (end_bit - begin_bit + r - 1) / r;
}

/* Digit p of a key: the bit field [lo, hi) with lo = begin + p*r. */
static uint64_t digit_of(uint64_t key, int begin_bit, int end_bit, int r, int p) {
  int lo = begin_bit + p * r;
  int hi = lo + r;
  if (hi > end_bit) hi = end_bit;
  int width = hi - lo;
  uint64_t mask = (width >= 64) ? ~0ull : ((1ull << width) - 1ull);
  return (key >> lo) & mask;
}

/* Step 1 of one counting sort: count[v] over all n elements. */
static void count_digits(const uint64_t* key, uint64_t n, int begin_bit, int end_bit,
                         int r, int p, uint64_t* count, uint64_t radix) {
  for (uint64_t v = 0; v < radix; ++v) count[v] = 0;
  for (uint64_t i = 0; i < n; ++i) count[digit_of(key[i], begin_bit, end_bit, r, p)] += 1;
}

/* Step 2: exclusive prefix sum, start[v] = sum_{u<v} count[u]. */
static void exclusive_prefix(const uint64_t* count, uint64_t* start, uint64_t radix) {
  uint64_t run = 0;
  for (uint64_t v = 0; v < radix; ++v) {
    start[v] = run;
    run += count[v];
  }
}

/*
 * The whole sort over 64-bit working copies of keys and values (narrower key
 * types are widened on entry and narrowed on exit, which changes no digit).
 */
static int lsd_sort_wide(uint64_t* key, uint64_t* val, uint64_t n, int key_bits,
                         int begin_bit, int end_bit, int r) {
  int passes = oracle_num_passes(key_bits, begin_bit, end_bit, r);
  if (passes < 0) return ORACLE_EINVAL;
  if (n < 2 || passes == 0) return ORACLE_OK;
  uint64_t radix = 1ull << r;
  uint64_t* count = (uint64_t*)malloc(radix * sizeof(uint64_t));
  uint64_t* start = (uint64_t*)malloc(radix * sizeof(uint64_t));
  uint64_t* key_out = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint64_t* val_out = val ? (uint64_t*)malloc(n * sizeof(uint64_t)) : NULL;
  if (!count || !start || !key_out || (val && !val_out)) {
    free(count); free(start); free(key_out); free(val_out);
    return ORACLE_ENOMEM;
  }
  for (int p = 0; p < passes; ++p) { /* least significant digit first */
    count_digits(key, n, begin_bit, end_bit, r, p, count, radix);
    exclusive_prefix(count, start, radix);
    for (uint64_t i = 0; i < n; ++i) { /* input order: stable */
      uint64_t v = digit_of(key[i], begin_bit, end_bit, r, p);
      uint64_t dst = start[v]++;
      key_out[dst] = key[i];
      if (val) val_out[dst] = val[i];
    }
    memcpy(key, key_out, n * sizeof(uint64_t));
    if (val) memcpy(val, val_out, n * sizeof(uint64_t));
  }
  free(count); free(start); free(key_out); free(val_out);
  return ORACLE_OK;
}

int oracle_lsd_sort_u64(uint64_t* keys, uint64_t* vals, uint64_t n, int begin_bit,
                        int end_bit, int r) {
  if (n && !keys) return ORACLE_EINVAL;
  return lsd_sort_wide(keys, vals, n, 64, begin_bit, end_bit, r);
}

int oracle_lsd_sort_u32(uint32_t* keys, uint32_t* vals, uint64_t n, int begin_bit,
                        int end_bit, int r) {
  if (n && !keys) return ORACLE_EINVAL;
  if (oracle_num_passes(32, begin_bit, end_bit, r) < 0) return ORACLE_EINVAL;
  if (n == 0) return ORACLE_OK;
  uint64_t* k = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint64_t* v = vals ? (uint64_t*)malloc(n * sizeof(uint64_t)) : NULL;
  if (!k || (vals && !v)) { free(k); free(v); return ORACLE_ENOMEM; }
  for (uint64_t i = 0; i < n; ++i) k[i] = keys[i];
  if (vals) for (uint64_t i = 0; i < n; ++i) v[i] = vals[i];
  int rc = lsd_sort_wide(k, v, n, 32, begin_bit, end_bit, r);
  if (rc == ORACLE_OK) {
    for (uint64_t i = 0; i < n; ++i) keys[i] = (uint32_t)k[i];
    if (vals) for (uint64_t i = 0; i < n; ++i) vals[i] = (uint32_t)v[i];
  }
  free(k); free(v);
  return rc;
}

/*
 * Digit histograms of every pass (step 1 of each counting sort, taken over
 * the input as given): counts[p * 2^r + v] = number of keys whose digit p
 * equals v.  The histogram of a digit does not depend on the order of the
 * keys, so these are also the counts each pass of the sort uses.
 */
int oracle_digit_counts_u64(const uint64_t* keys, uint64_t n, int key_bits, int begin_bit,
                            int end_bit, int r, uint64_t* counts) {
  int passes = oracle_num_passes(key_bits, begin_bit, end_bit, r);
  if (passes < 0 || (n && !keys) || !counts) return ORACLE_EINVAL;
  uint64_t radix = 1ull << r;
  for (int p = 0; p < passes; ++p)
    count_digits(keys, n, begin_bit, end_bit, r, p, counts + (uint64_t)p * radix, radix);
  return ORACLE_OK;
}

/* Exclusive prefix of each pass's histogram (step 2), same layout. */
int oracle_digit_offsets(const uint64_t* counts, int passes, int r, uint64_t* offsets) {
  if (passes < 0 || r < 1 || r > 16 || !counts || !offsets) return ORACLE_EINVAL;
  uint64_t radix = 1ull << r;
  for (int p = 0; p < passes; ++p)
    exclusive_prefix(counts + (uint64_t)p * radix, offsets + (uint64_t)p * radix, radix);
  return ORACLE_OK;
}

/*
 * Segmented variant: the same sort applied independently to every segment
 * [offsets[s], offsets[s+1]) of one array, s = 0 .. nseg-1.
 */
int oracle_segmented_sort_u32(uint32_t* keys, uint32_t* vals, const uint64_t* offsets,
                              uint64_t nseg, int begin_bit, int end_bit, int r) {
  if (nseg && !offsets) return ORACLE_EINVAL;
  for (uint64_t s = 0; s < nseg; ++s) {
    if (offsets[s + 1] < offsets[s]) return ORACLE_EINVAL;
    uint64_t len = offsets[s + 1] - offsets[s];
    int rc = oracle_lsd_sort_u32(keys + offsets[s], vals ? vals + offsets[s] : NULL, len,
                                 begin_bit, end_bit, r);
    if (rc) return rc;
  }
  return ORACLE_OK;
}

int oracle_segmented_sort_u64(uint64_t* keys, uint64_t* vals, const uint64_t* offsets,
                              uint64_t nseg, int begin_bit, int end_bit, int r) {
  if (nseg && !offsets) return ORACLE_EINVAL;
  for (uint64_t s = 0; s < nseg; ++s) {
    if (offsets[s + 1] < offsets[s]) return ORACLE_EINVAL;
    uint64_t len = offsets[s + 1] - offsets[s];
    int rc = oracle_lsd_sort_u64(keys + offsets[s], vals ? vals + offsets[s] : NULL, len,
                                 begin_bit, end_bit, r);
    if (rc) return rc;
  }
  return ORACLE_OK;
}

/*
 * Key orders beyond the paper's unsigned keys.  The order key of a w-bit
 * pattern is an unsigned w-bit integer whose ascending order is the wanted
 * order; the sort then orders the order keys (the LSD sort above) and
 * carries the original patterns along.  Written from the definitions:
 *   kind 0, unsigned: the pattern's value.
 *   kind 1, two's complement: value v in [-2^(w-1), 2^(w-1)), order key
 *           v + 2^(w-1).
 *   kind 2, IEEE-754 (binary32 for w = 32, binary64 for w = 64): sign s and
 *           the remaining bits m (exponent and fraction, which order the
 *           magnitudes); IEEE totalOrder puts every negative pattern below
 *           every positive one and orders negatives by decreasing m:
 *           order key = 2^(w-1) - 1 - m if s, else 2^(w-1) + m.
 *   descending: the order key u becomes (2^w - 1) - u.
 */
static uint64_t order_key(uint64_t bits, int w, int kind, int descending) {
  const uint64_t half = (uint64_t)1 << (w - 1);
  const uint64_t all = half + (half - 1);  /* 2^w - 1 */
  uint64_t u;
  if (kind == 0) {
    u = bits;
  } else if (kind == 1) {
    /* patterns >= 2^(w-1) hold v = pattern - 2^w, so v + 2^(w-1) = pattern - 2^(w-1) */
    u = bits >= half ? bits - half : bits + half;
  } else {
    const uint64_t m = bits & (half - 1);
    u = (bits & half) ? half - 1 - m : half + m;
  }
  return descending ? all - u : u;
}

int oracle_order_keys_u32(const uint32_t* keys, uint32_t* out, uint64_t n, int kind,
                          int descending) {
  if ((n && (!keys || !out)) || kind < 0 || kind > 2) return ORACLE_EINVAL;
  for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)order_key(keys[i], 32, kind, descending);
  return ORACLE_OK;
}

int oracle_order_keys_u64(const uint64_t* keys, uint64_t* out, uint64_t n, int kind,
                          int descending) {
  if ((n && (!keys || !out)) || kind < 0 || kind > 2) return ORACLE_EINVAL;
  for (uint64_t i = 0; i < n; ++i) out[i] = order_key(keys[i], 64, kind, descending);
  return ORACLE_OK;
}
