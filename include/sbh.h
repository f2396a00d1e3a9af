/*
 * sbh.h -- C ABI of the KPA grouping path (StreamBox-HBM, Miao et al.,
 * ASPLOS '19), built for NVIDIA B300 (sm_103a).
 *
 * A Key Pointer Array (KPA, Sec. 4.1) is held as two device arrays of equal
 * length n: keys (uint64, the resident key) and ptrs (uint32, the row index
 * of the full record in its columnar stream).  The canonical order of a
 * sorted KPA is (key ascending, ptr ascending).
 *
 * Common rules for every call below:
 *  - Pointers named d_* are device pointers (cudaMalloc / PyTorch CUDA
 *    memory) owned by the caller.  The library never frees or keeps them.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream).  A call returns once its kernels are queued.
 *  - Calls that need working memory take (d_scratch, scratch_bytes).  With
 *    d_scratch == NULL the call only stores the required size in
 *    *scratch_bytes and returns SBH_OK without touching the GPU.  Otherwise
 *    *scratch_bytes must be at least that size.  Scratch must be 256-byte
 *    aligned, must not overlap inputs or outputs, and may be reused once the
 *    call's work on `stream` has finished.  Two calls that run at the same
 *    time need two scratch buffers.
 *  - Inputs are never written.
 *  - Counts that depend on the data (distinct keys, join pairs) are written
 *    to a caller-supplied device uint64; outputs beyond the caller's
 *    capacity are not written, but the full count is still stored, so the
 *    caller can compare it with the capacity after synchronising.
 *  - Return values: SBH_OK, or a host-side error detected before any launch
 *    (SBH_EINVAL: bad argument; SBH_ENOSPACE: scratch too small; SBH_ECUDA:
 *    a CUDA runtime error, text in sbh_last_error()).  Nothing aborts,
 *    throws or traps.
 *  - Device-side waits (decoupled look-back between tiles) are bounded.  A
 *    wait that runs out records SBH_ETIMEOUT in a per-device status word
 *    that sbh_sync_status() reads; the call's output is then invalid.
 */
#ifndef SBH_H
#define SBH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBH_OK 0
#define SBH_EINVAL 1
#define SBH_ENOSPACE 2
#define SBH_ETIMEOUT 3
#define SBH_ECUDA 4

/* Unused top-K slots hold this value and pointer. */
#define SBH_TOPK_PAD_VAL 0ull
#define SBH_TOPK_PAD_PTR 0xFFFFFFFFu
#define SBH_TOPK_MAX_K 8

/* Library version string. */
const char* sbh_version(void);

/* Text of the last host-side error on the calling thread ("" if none). */
const char* sbh_last_error(void);

/* Wait for `stream`, then return SBH_OK, or SBH_ETIMEOUT if any kernel of
 * this library on the current device recorded an expired device-side wait
 * since the last call (the record is cleared), or SBH_ECUDA on a CUDA error. */
int sbh_sync_status(void* stream);

/* Test hooks.  sbh_set_spin_limit sets the number of polls a device-side
 * wait makes before it gives up (0 restores the default).
 * sbh_set_fault(SBH_FAULT_SKIP_PUBLISH) makes every pass of the next
 * sbh_kpa_sort call leave tile 0's look-back record unpublished, so that the
 * waits of later tiles run out (n must exceed one tile of 4096 keys); it is
 * cleared by that call.  Neither hook faults or hangs the device. */
#define SBH_FAULT_NONE 0
#define SBH_FAULT_SKIP_PUBLISH 1
void sbh_set_spin_limit(uint32_t polls);
void sbh_set_fault(int fault);

/* Per-launch timing.  sbh_profile_enable(1) clears earlier records and
 * makes every later call record a CUDA event pair around each of its kernel
 * launches, on the launch's stream; sbh_profile_enable(0) stops recording
 * (and also clears).  sbh_profile_collect waits for the recorded events and
 * copies, for the first max_records launches in launch order, the kernel name
 * (names + i * name_len, NUL-terminated, truncated to name_len - 1 bytes) and
 * its duration in milliseconds (ms[i]); either buffer may be NULL.  It
 * returns the number of records. */
/* Tuning knobs, process-wide, read by every later call (the autotuner in
 * the Python package measures and sets them; the defaults are measured on
 * B300):
 *   SBH_KNOB_SORT_CHUNKED_MIN        sorts of at least this many pairs take
 *                                    per-chunk count / scan / scatter passes,
 *                                    smaller ones one onesweep kernel a pass
 *                                    (default 2^23);
 *   SBH_KNOB_MERGE_SEARCH_MIN_TILES  merges of more than this many 2048-row
 *                                    output tiles find the tiles' cuts in a
 *                                    separate parallel search (default 2047);
 *   SBH_KNOB_SCATTER_GEOM            tile and CTA of the plain sort's chunked
 *                                    scatter: 0 = 4096 rows, 512 threads,
 *                                    two CTAs per SM (default); 1 = 2048
 *                                    rows, 256 threads, four; 2 = 8192 rows,
 *                                    1024 threads, one.
 * A sort's scratch size depends on the first knob: size it after setting.
 * sbh_set_knob returns SBH_EINVAL for an unknown knob or an out-of-range
 * geometry; sbh_get_knob 0 for an unknown knob. */
#define SBH_KNOB_SORT_CHUNKED_MIN 0
#define SBH_KNOB_MERGE_SEARCH_MIN_TILES 1
#define SBH_KNOB_SCATTER_GEOM 2
#define SBH_KNOB_COUNT 3
int sbh_set_knob(int knob, uint64_t value);
uint64_t sbh_get_knob(int knob);

void sbh_profile_enable(int on);
int sbh_profile_collect(int max_records, char* names, int name_len, double* ms);

/* ---------------------------------------------------------------- A1
 * Window ranges (Sec. 4.2 "Windowing": Partition on the timestamp column).
 * Window w holds the rows whose timestamp lies in [d_starts[w], d_starts[w]
 * + len).  d_ts (n values of ts_bytes = 4 or 8 bytes) must be
 * non-decreasing and d_starts[w] + len below 2^64; each window is the row
 * range [d_row_begin[w],
 * d_row_end[w]), found by binary search.  No scratch. */
int sbh_window_ranges(const void* d_ts, int ts_bytes, uint64_t n, const uint64_t* d_starts, uint64_t len,
                      uint64_t nwin, uint64_t* d_row_begin, uint64_t* d_row_end, void* stream);

/* ---------------------------------------------------------------- A2
 * Extract (Table 2; Sec. 4.2 "Maintenance primitives": copy the key column
 * and initialise the record pointers).  For i < n:
 *     d_keys[i] = key_col[row_begin + i],  d_ptrs[i] = row_begin + i.
 * key_col may be device memory or page-locked host memory (cudaHostAlloc /
 * cudaHostRegister); in the latter case the kernel reads it over the host
 * link.  row_begin + n must be < 2^32.
 * Optional by-products (pass NULL to skip):
 *   d_key_or   one uint64: bitwise OR of the n keys (significant bits).
 *   d_samples  ceil(n / sample_stride) keys: d_samples[j] = d_keys[j*stride].
 * With d_keys and d_ptrs both NULL (and d_key_or NULL) only the samples are
 * written, read straight from the column: the sample a learned sort of the
 * column trains on when the sort reads the column itself (see
 * sbh_kpa_sort).
 * No scratch. */
int sbh_kpa_extract(const uint64_t* key_col, uint64_t row_begin, uint64_t n, uint64_t* d_keys, uint32_t* d_ptrs,
                    uint64_t* d_key_or, uint64_t* d_samples, uint64_t sample_stride, void* stream);

/* Extract of many tumbling windows at once (Sec. 4.2 "Windowing": records
 * are partitioned into windows; the paper gives no batched form, which is
 * this library's design).  Window w holds rows [d_offsets[w], d_offsets[w +
 * 1]) of key_col; d_offsets (device, nwin + 1 non-decreasing values) covers
 * rows [row_begin, row_begin + n) = [d_offsets[0], d_offsets[nwin]).  For
 * i < n, row r = row_begin + i of window w gives
 *     d_keys[i] = (w << (64 - sbh_window_bits(nwin))) | key_col[r],
 *     d_ptrs[i] = r.
 * Sorting these composite keys orders the rows by (window, key, ptr), so one
 * sort, one keyed reduction and one top-K serve every window, and the
 * results of window w are the output keys in [w << shift, (w + 1) << shift)
 * (found with sbh_window_ranges).  The composite is exact only when every
 * key is below 2^(64 - sbh_window_bits(nwin)); d_key_or (nullable, device)
 * receives the OR of the raw keys so that the caller can check.  key_col may
 * be device memory or page-locked host memory.  No scratch. */
int sbh_kpa_extract_windows(const uint64_t* key_col, const uint64_t* d_offsets, uint64_t nwin, uint64_t row_begin,
                            uint64_t n, uint64_t* d_keys, uint32_t* d_ptrs, uint64_t* d_key_or, void* stream);
/* Bits of the window field of the composite keys: the bit length of nwin. */
int sbh_window_bits(uint64_t nwin);

/* Split of an arriving bundle into window slots by timestamp (Sec. 4.2
 * "Windowing": records belong to the window of their timestamp; Sec. 3
 * watermarks decide when a window closes).  Row i of the bundle (device
 * columns key_col[i], ts_rel[i], i < n) has timestamp ts_base + ts_rel[i]
 * and window w = timestamp / win_len.  Rows of window first_win or
 * first_win + 1 are appended, in row order, to slot w & 1: pairs
 * (key_col[i], ptr_base + i) go to (d_keys0, d_ptrs0) or (d_keys1,
 * d_ptrs1) at index d_fill[slot] onwards, and d_fill[slot] (device, two
 * uint64) moves on; other rows (late, or more than one window ahead, or a
 * negative timestamp) are dropped and added to *d_dropped.  A slot never
 * grows past cap0 / cap1: the rows that do not fit are not written and
 * *d_overflow is set to 1.  Several bundles in a row on one stream append
 * after one another; no host synchronisation is needed.
 * Scratch: 12 bytes per 4096 rows. */
int sbh_kpa_split_ts(const uint64_t* key_col, const int64_t* ts_rel, uint64_t n, int64_t ts_base, uint64_t win_len,
                     uint64_t first_win, uint32_t ptr_base, uint64_t* d_keys0, uint32_t* d_ptrs0, uint64_t cap0,
                     uint64_t* d_keys1, uint32_t* d_ptrs1, uint64_t cap1, uint64_t* d_fill, uint64_t* d_dropped,
                     uint32_t* d_overflow, void* d_scratch, size_t* scratch_bytes, void* stream);

/* ---------------------------------------------------------------- A3
 * Sort (Table 2: order a KPA by its resident key).  Stable LSD radix sort,
 * 8-bit digits, one pass per digit position whose digit is not the same for
 * all keys (the histogram of every position is built in one read).  Below
 * 2^23 pairs (SBH_KNOB_SORT_CHUNKED_MIN) each pass is one onesweep kernel: tile load, warp multisplit
 * ranking, decoupled look-back for the tile's global digit offsets, scatter
 * staged through shared memory.  From 2^23 pairs each pass is three kernels:
 * per-chunk digit counts, their scan, and a scatter in which every CTA walks
 * its own chunk of tiles (bulk-copied, ranked, staged) with its digit offsets
 * known up front; each scatter also stores every row's digit of the next
 * pass (one byte), which that pass's chunk counts read instead of the keys.
 * Because the sort is stable and ties keep their input
 * order, the output is in (key, ptr) order when the input ptrs ascend (as
 * Extract makes them); in general ties keep input order.
 * In/out: (d_keys_in, d_ptrs_in) -> (d_keys_out, d_ptrs_out), n pairs,
 * n < 2^32.  The output may alias the input (in-place sort).
 * d_ptrs_in may be NULL (not in place): input row i's ptr is then i.  A
 * resident key column is sorted this way without an Extract pass: the first
 * digit pass reads the column and makes each ptr from its row number, and
 * the output is what Extract (row_begin 0) followed by this sort gives.
 * Scratch: about 13 n bytes plus 2 MiB (the sizing call gives the exact figure). */
int sbh_kpa_sort(const uint64_t* d_keys_in, const uint32_t* d_ptrs_in, uint64_t* d_keys_out, uint32_t* d_ptrs_out,
                 uint64_t n, void* d_scratch, size_t* scratch_bytes, void* stream);

/* ---------------------------------------------------------------- A5
 * Merge (Table 2: merge sorted KPAs; Sec. 4.2 "Keyed Aggregation" merges the
 * sorted KPAs of a window when it closes).  nruns sorted runs, each in (key,
 * ptr) order, are merged into one run in (key, ptr) order by rounds of
 * pairwise merge-path merges.  Host arrays d_run_keys[r], d_run_ptrs[r]
 * hold device pointers; run_lens[r] is a host array.  Total length < 2^32.
 * Scratch: 4 bytes per 2048 output pairs, plus 24 * total bytes when nruns > 2. */
int sbh_kpa_merge(int nruns, const uint64_t* const* d_run_keys, const uint32_t* const* d_run_ptrs,
                  const uint64_t* run_lens, uint64_t* d_keys_out, uint32_t* d_ptrs_out, void* d_scratch,
                  size_t* scratch_bytes, void* stream);

/* Many independent merges in one pass (Sec. 4.2 "Temporal Join" merges
 * the sorted KPAs of each window; with sliding windows built from panes,
 * every window merges its panes, and all windows are merged at once here).
 * Segment g merges A rows [a_start[g], a_start[g] + a_len[g]) of (d_a_keys,
 * d_a_ptrs) with B rows [b_start[g], b_start[g] + b_len[g]) of (d_b_keys,
 * d_b_ptrs), each sorted in (key, ptr) order, into (key, ptr) order; the
 * segments' outputs lie end to end in (d_keys_out, d_ptrs_out) in segment
 * order.  The four segment arrays are host arrays of nseg values; segments
 * may overlap in the inputs (A and B may be the same arrays); every row
 * index and the total output stay below 2^32.  Two kernels: the co-rank of
 * every output tile (a binary search per 2048-row tile) and the merge path
 * of every tile.  The output must not overlap the inputs.
 * Scratch: 48 bytes per segment plus 4 bytes per 2048 output rows. */
int sbh_kpa_merge_segments(int nseg, const uint64_t* d_a_keys, const uint32_t* d_a_ptrs, const uint64_t* d_b_keys,
                           const uint32_t* d_b_ptrs, const uint64_t* a_start, const uint64_t* a_len,
                           const uint64_t* b_start, const uint64_t* b_len, uint64_t* d_keys_out,
                           uint32_t* d_ptrs_out, void* d_scratch, size_t* scratch_bytes, void* stream);

/* ---------------------------------------------------------------- A6
 * Keyed reduction (Table 2; Sec. 4.2 "Reduction primitives": scan a sorted
 * KPA, find each contiguous key range, and coalesce a nonresident column
 * reached through the pointers).  For each distinct key, in key order:
 *   d_out_keys[j]   the key,
 *   d_out_counts[j] its number of records, count_bytes = 4 or 8 bytes each
 *                   (a count is below 2^32, so 4 bytes always hold it),
 *   d_out_sums[j]   the sum of d_val_col[ptr] over its records, modulo 2^64
 *                   (d_val_col has val_bytes = 4 or 8 bytes per row).
 * d_val_col == NULL (or d_out_sums == NULL) computes counts only and reads
 * no values.  *d_nkeys receives the number of distinct keys; only the first
 * cap entries are written.  The input must be sorted by key.
 * Scratch: about 64 * (n / 4096) bytes. */
int sbh_group_reduce(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col,
                     int val_bytes, uint64_t* d_out_keys, void* d_out_counts, int count_bytes, uint64_t* d_out_sums,
                     uint64_t cap, uint64_t* d_nkeys, void* d_scratch, size_t* scratch_bytes, void* stream);

/* The keyed reduction above without the scratch argument, for callers that
 * cannot allocate device memory when they call: a serving loop that fixes
 * its device memory at start-up (cudaMalloc may also synchronise the device
 * and stall other streams), or a host that hands this library only its
 * input and output buffers.  The paper has no counterpart; it is an
 * interface of this library.
 * Arguments and results are those of sbh_group_reduce; n is at most 2^28
 * rows, and a larger n returns SBH_EINVAL without launching.  Its working
 * memory is one fixed device array of just over 2 MiB, which every GPU that
 * loads the library holds until the process exits; the call allocates and frees
 * nothing.  The first call on a device looks up that array's device address
 * (once per device, with that device current), so make that first call
 * before any stream capture.  All calls on a device share the array and it
 * keeps the last call's contents (nothing in it needs to start at zero): two
 * calls whose work overlaps on the GPU race and give wrong results, so
 * serialise them, e.g. on one stream. */
int sbh_group_reduce_noalloc(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col,
                             int val_bytes, uint64_t* d_out_keys, void* d_out_counts, int count_bytes,
                             uint64_t* d_out_sums, uint64_t cap, uint64_t* d_nkeys, void* stream);

/* ---------------------------------------------------------------- A7
 * Top-K per key (Sec. 7, benchmark 1 "TopK Per Key": the K largest values of
 * each key).  For each distinct key j, in key order, the min(K, count)
 * records with the largest d_val_col[ptr], ordered by (value descending, ptr
 * ascending): d_out_vals[j*K + s], d_out_ptrs[j*K + s] for s < K, unused
 * slots padded with SBH_TOPK_PAD_VAL / SBH_TOPK_PAD_PTR; d_out_nvalid[j] =
 * min(K, count).  1 <= K <= SBH_TOPK_MAX_K.  Input sorted by key; cap and
 * *d_nkeys as in sbh_group_reduce; n < 2^32 - 1.  The keys' runs are found
 * first; runs of at most 64 rows are reduced by one thread each, runs of up
 * to 4096 rows by one warp each, longer ones in chunks of 16384 rows by one
 * CTA each, no CTA waiting on another.
 * Scratch: about 4 n bytes. */
int sbh_topk(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col, int val_bytes,
             int K, uint64_t* d_out_keys, uint8_t* d_out_nvalid, uint64_t* d_out_vals, uint32_t* d_out_ptrs,
             uint64_t cap, uint64_t* d_nkeys, void* d_scratch, size_t* scratch_bytes, void* stream);

/* Median and distinct values per key (Sec. 7, benchmarks "Median" and
 * "Unique Count"; Average is sum / count from sbh_group_reduce).  For each
 * distinct key j of a KPA sorted by key, in key order: d_out_keys[j],
 * d_out_median[j] = the lower median of its values d_val_col[ptr] (the value
 * at index (count - 1) / 2 of the key's values in ascending order), and
 * d_out_unique[j] = the number of distinct values.  The rows are re-ordered
 * by (key, value) with two stable radix sorts (by value, then by key), so
 * inside each key's run the values ascend.  val_bytes 4 or 8; cap and
 * *d_nkeys as in sbh_group_reduce; n < 2^32 - 1.
 * Scratch: about 70 n bytes. */
int sbh_median_unique(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_val_col,
                      int val_bytes, uint64_t* d_out_keys, uint64_t* d_out_median, uint64_t* d_out_unique,
                      uint64_t cap, uint64_t* d_nkeys, void* d_scratch, size_t* scratch_bytes, void* stream);

/* Materialize (Table 2: the values of a column for the records of a KPA, in
 * KPA order): d_out[i] = d_col[d_ptrs[i]] for i < n, col_bytes 4 or 8 (d_out
 * holds n such values).  n < 2^32.  No scratch. */
int sbh_kpa_materialize(const uint32_t* d_ptrs, uint64_t n, const void* d_col, int col_bytes, void* d_out,
                        void* stream);

/* KeySwap (Table 2: make another key column the KPA's resident key):
 * d_keys_out[i] = d_key_col[d_ptrs[i]]; the pointers are unchanged, and the
 * new KPA (d_keys_out, d_ptrs) is in the old key order until it is sorted
 * again.  No scratch. */
int sbh_kpa_keyswap(const uint32_t* d_ptrs, uint64_t n, const uint64_t* d_key_col, uint64_t* d_keys_out,
                    void* stream);

/* KeySwap through a lookup table (Sec. 4.2: Materialize of a column fused
 * with the Extract of the new key, as when a pipeline maps each record's ad
 * to its campaign before grouping): d_keys_out[i] = d_table[v] with v =
 * d_col[d_ptrs[i]] when v < table_len; otherwise d_keys_out[i] = ~0 and the
 * row is added to *d_misses (device, nullable).  Pointers are unchanged.
 * No scratch. */
int sbh_kpa_keyswap_lookup(const uint32_t* d_ptrs, uint64_t n, const uint64_t* d_col, const uint64_t* d_table,
                           uint64_t table_len, uint64_t* d_keys_out, uint64_t* d_misses, void* stream);

/* Counted copy: dst[i] = d_src[i] for i < min(*d_count, cap) * per, with
 * elements of elem_bytes = 1, 4 or 8 bytes, where the count is known only on
 * the device (the number of distinct keys a reduction wrote).  dst_bytes is
 * elem_bytes, or 4 with elem_bytes 8: each value is stored as its low 4
 * bytes (per-key counts, which are below 2^32, copied back in half the
 * bytes).  dst may be
 * page-locked host memory (cudaHostAlloc / cudaHostRegister), written by the
 * kernel over the host link, so that a window's per-key results reach the
 * host without a host synchronisation between the reduction and the copy
 * (Sec. 4.2 "Keyed Aggregation" emits them when the window closes).  The
 * paper has no such primitive; it is plumbing of this library.  No scratch. */
int sbh_copy_counted(const void* d_src, void* dst, int elem_bytes, int dst_bytes, const uint64_t* d_count,
                     uint64_t per, uint64_t cap, void* stream);

/* Select (Table 2: filter the records of a KPA): the pairs whose value
 * d_col[ptr] (col_bytes 4 or 8) lies in [lo, hi), in KPA order, to
 * (d_out_keys, d_out_ptrs); *d_count (device) receives how many and only the
 * first cap are written.  n < 2^32.
 * Scratch: 4 bytes per 4096 rows. */
int sbh_kpa_select(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const void* d_col, int col_bytes,
                   uint64_t lo, uint64_t hi, uint64_t* d_out_keys, uint32_t* d_out_ptrs, uint64_t cap,
                   uint64_t* d_count, void* d_scratch, size_t* scratch_bytes, void* stream);

/* Partition (Table 2: split a KPA into sub-KPAs by ranges of its resident
 * keys; Sec. 4.2 "Windowing" applies it to the timestamp column).  d_bounds
 * (device, nb non-decreasing keys, nb < 2^32 - 1) cut the key space into
 * nb + 1 ranges: part j holds the pairs with d_bounds[j - 1] <= key <
 * d_bounds[j] (no lower limit for part 0, no upper limit for part nb).  The
 * input KPA (n < 2^32 pairs, any order) is written to (d_keys_out,
 * d_ptrs_out) part after part, each part in the input order, and
 * d_offsets[j] (device, nb + 2 uint64) receives the first row of part j,
 * d_offsets[nb + 1] = n.  The output may alias the input (both arrays).
 * It is a stable sort by part number: one 8-bit radix pass for up to 256
 * parts, two for up to 65536, and so on.
 * Scratch: that of sbh_kpa_sort for n pairs. */
int sbh_kpa_partition(const uint64_t* d_keys, const uint32_t* d_ptrs, uint64_t n, const uint64_t* d_bounds,
                      uint64_t nb, uint64_t* d_keys_out, uint32_t* d_ptrs_out, uint64_t* d_offsets, void* d_scratch,
                      size_t* scratch_bytes, void* stream);

/* ---------------------------------------------------------------- A8
 * Join (Table 2: join two sorted KPAs by resident key; Sec. 4.2 "Temporal
 * Join" joins the KPAs of one window of each stream).  Emits every pair
 * (ptrL, ptrR) with keyL == keyR, in (key, ptrL, ptrR) order, into
 * d_out_l[p], d_out_r[p].  Both inputs sorted in (key, ptr) order.
 * *d_npairs receives the number of pairs; only the first cap are written.
 * Scratch: about 16 * nl bytes. */
int sbh_join(const uint64_t* d_lkeys, const uint32_t* d_lptrs, uint64_t nl, const uint64_t* d_rkeys,
             const uint32_t* d_rptrs, uint64_t nr, uint32_t* d_out_l, uint32_t* d_out_r, uint64_t cap,
             uint64_t* d_npairs, void* d_scratch, size_t* scratch_bytes, void* stream);

/* Many independent joins in one pass (Sec. 4.2 "Temporal Join", every
 * window of a sliding-window join at once).  Segment g joins L rows
 * [l_off[g], l_off[g + 1]) of (d_lkeys, d_lptrs) with R rows [r_start[g],
 * r_start[g] + r_len[g]) of (d_rkeys, d_rptrs), each sorted in (key, ptr)
 * order; the pairs of segment g, in (key, ptrL, ptrR) order, are output rows
 * [d_seg_pairs[g], d_seg_pairs[g + 1]) of (d_out_l, d_out_r).  l_off (host,
 * nseg + 1 non-decreasing values from 0), r_start and r_len (host, nseg
 * values) describe the segments; R segments may overlap.  *d_npairs and
 * d_seg_pairs[nseg] receive the total; only the first cap pairs are
 * written (cap 0: only the counts).  reuse_counts != 0: the scratch holds
 * the counts of an earlier call with the same inputs and segments (made
 * with cap 0 to size the output), and only the pairs are written (the
 * matches are not searched again).  L below 2^32 rows.
 * Scratch: about 8 bytes per L row plus 24 bytes per segment. */
int sbh_join_segments(int nseg, const uint64_t* d_lkeys, const uint32_t* d_lptrs, const uint64_t* l_off,
                      const uint64_t* d_rkeys, const uint32_t* d_rptrs, const uint64_t* r_start,
                      const uint64_t* r_len, uint32_t* d_out_l, uint32_t* d_out_r, uint64_t cap,
                      uint64_t* d_npairs, uint64_t* d_seg_pairs, int reuse_counts, void* d_scratch,
                      size_t* scratch_bytes, void* stream);

/* ---------------------------------------------------------------- A4
 * Learned MSD partition sort.  The paper has no learned component (its Sort
 * splits a KPA into chunks sorted in-core, Sec. 4.2 "Primitive
 * Implementation"); this path produces exactly the output of sbh_kpa_sort.
 *
 * The network is a 1-32-32-1 ReLU MLP in FP32 with SBH_MLP_PARAMS parameters
 * laid out as W1[32], b1[32], W2[32][32] (row = output unit), b2[32],
 * w3[32], b3.  Its input is a key's feature x(k) = (m + f / 2^17) / 64, m the
 * index of the highest set bit and f the 17 bits below it (x(0) = 0). */
#define SBH_MLP_PARAMS 1153
#define SBH_LEARNED_MODEL_BYTES 139264
#define SBH_LEARNED_CAPACITY 8192 /* rows a bucket may hold to be sorted in shared memory */
#define SBH_LEARNED_MAX_HEAVY 16384 /* heavy keys a model holds */
#define SBH_LEARNED_STATS 14

/* y[i] = MLP(x[i]) for i < m.  No scratch. */
int sbh_mlp_forward(const float* d_params, const float* d_x, uint64_t m, float* d_y, void* stream);

/* Gradient of the mean squared error (1/m) sum_i (MLP(x[i]) - t[i])^2 with
 * respect to the parameters into d_grad (SBH_MLP_PARAMS floats), and the
 * loss into *d_loss (nullable).  Sums run in a fixed order, so repeated
 * calls give identical results.  Scratch: about 4.6 KB per 256 rows. */
int sbh_mlp_grad(const float* d_params, const float* d_x, const float* d_t, uint64_t m, float* d_grad,
                 float* d_loss, void* d_scratch, size_t* scratch_bytes, void* stream);

/* Fits a model to a key sample (d_samples, m keys standing for n_rows rows,
 * e.g. every 100th row from sbh_kpa_extract).  Steps:
 *  1. sort the sample;
 *  2. heavy keys: a key value whose sample count times n_rows exceeds
 *     (SBH_LEARNED_CAPACITY / 2) times m gets a dedicated bucket (the
 *     smallest SBH_LEARNED_MAX_HEAVY such keys, if there are more); its
 *     samples leave the training set;
 *  3. training set of m' rows: row r takes the sorted non-heavy sample
 *     j = (r * P) mod m' (P = first integer >= 2654435761 mod m' coprime
 *     with m'), input x(key), target (#samples < key + #samples <= key) / 2m';
 *  4. `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, rate lr) on batches of
 *     `batch` rows, step j using rows (j * batch + q) mod m', starting from
 *     d_init_params, or, when it is NULL, from the network that interpolates
 *     the training set's CDF linearly between 33 quantiles (knot i: sorted
 *     non-heavy sample floor(i (m' - 1) / 32), at its feature and CDF target;
 *     knots of equal feature merge, keeping the later target; first-layer
 *     unit u kinks at knot u, the second layer is the identity, the output
 *     weights are the changes of slope).  batch is a multiple of 128, at most
 *     32768.
 * d_model (SBH_LEARNED_MODEL_BYTES, device) receives the weights and the
 * heavy keys (ascending).  d_losses (nullable, `steps` floats) receives each
 * step's batch loss before its update; d_train_x / d_train_t (nullable, m
 * floats each) receive the training set (the first m' entries are
 * meaningful).
 * Scratch: about 32 m bytes plus the sort scratch for m. */
int sbh_learned_train(const uint64_t* d_samples, uint64_t m, uint64_t n_rows, const float* d_init_params,
                      int steps, int batch, float lr, void* d_model, float* d_losses, float* d_train_x,
                      float* d_train_t, void* d_scratch, size_t* scratch_bytes, void* stream);

/* Sorts a KPA with the model: bucket ids from the model's CDF (monotone in
 * the key by construction), a stable scatter by bucket id, a shared-memory
 * sort of every bucket of at most SBH_LEARNED_CAPACITY rows and more than one
 * key, and the plain radix sort for the rows of larger buckets.  Every step
 * is stable, so the output is identical to sbh_kpa_sort's for any ptrs (ties
 * keep their input order); input and output must not alias.  d_ptrs_in may
 * be NULL, as for sbh_kpa_sort: row i's ptr is i (the key column sorted
 * without an Extract pass; train on the column's samples, see
 * sbh_kpa_extract).  Like every call
 * here it only queues work on `stream`: the bucket count, the heavy keys in
 * use and the number of rows left to the plain radix sort are settled on the
 * device.  (When every bucket id fits in 16 bits, the ids travel with the
 * rows; if the model's heavy keys would push ids past that, only the
 * smallest of them keep a bucket of their own.)
 * Consecutive buckets of at most SBH_LEARNED_CAPACITY rows together are
 * sorted in shared memory as one run.
 * d_stats (nullable, device, SBH_LEARNED_STATS uint64 values, written by
 * the call's last kernel): bucket ids, heavy keys used, buckets sorted in
 * shared memory, one-key buckets (in runs of one key), heavy buckets,
 * overflow buckets, overflow rows, largest bucket, buckets sorted by radix
 * passes in shared memory (their runs were too uneven for the counting
 * placement) and their rows, and wide buckets and their rows (too uneven,
 * with a key range wider than 2^40, and a repeated key sharing its 16-bit
 * group of the key with another key even in a run of its bucket alone: they
 * join the overflow rows in the plain radix sort, cheaper than six or more
 * passes in shared memory), the buckets of runs whose group sort failed
 * and that were retried bucket by bucket, and the scatter passes on the
 * 16-bit bucket ids that ran (bit 0: the low byte, bit 1: the high byte; 0
 * when the ids were wider than 16 bits and not carried).
 * Scratch: about 24 n bytes. */
int sbh_kpa_sort_learned(const uint64_t* d_keys_in, const uint32_t* d_ptrs_in, uint64_t* d_keys_out,
                         uint32_t* d_ptrs_out, uint64_t n, const void* d_model, uint64_t* d_stats, void* d_scratch,
                         size_t* scratch_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SBH_H */
