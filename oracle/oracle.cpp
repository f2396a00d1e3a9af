/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, obviously correct CPU statement of what the KPA grouping
 * path computes (StreamBox-HBM, Sec. 4.1 "KPA" and Sec. 4.2 "Streaming
 * Operations", Table 2).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * Conventions (the readings the CUDA path must reproduce bit for bit):
 *   - A KPA is a pair of arrays keys[u64], ptrs[u32]; ptr is a row index.
 *   - The canonical order of a KPA is (key ascending, ptr ascending).
 *   - Sums are u64 and wrap modulo 2^64; counts are u64.
 *   - Top-K keeps, per key, the min(K, count) records with the largest value,
 *     ordered by (value descending, ptr ascending); unused slots hold value 0
 *     and ptr 0xFFFFFFFF.
 *   - Join emits every (ptrL, ptrR) with keyL == keyR, ordered by
 *     (key, ptrL, ptrR).
 *   - A window is the half-open timestamp range [start, start + len).
 */
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

namespace {

uint64_t load_val(const void* col, int bytes, uint64_t i) {
    return bytes == 8 ? static_cast<const uint64_t*>(col)[i] : static_cast<const uint32_t*>(col)[i];
}

uint64_t load_ts(const void* col, int bytes, uint64_t i) {
    return bytes == 8 ? static_cast<const uint64_t*>(col)[i] : static_cast<const uint32_t*>(col)[i];
}

}  // namespace

extern "C" {

/* Extract (Table 2; Sec. 4.2, "Maintenance primitives"): copy the key column
 * of rows [row_begin, row_begin + n) and set each pointer to its row. */
void oracle_extract(const uint64_t* key_col, uint64_t row_begin, uint64_t n, uint64_t* keys, uint32_t* ptrs) {
    for (uint64_t i = 0; i < n; ++i) {
        keys[i] = key_col[row_begin + i];
        ptrs[i] = static_cast<uint32_t>(row_begin + i);
    }
}

/* Sort (Table 2): order the KPA by resident key; ties by pointer. */
void oracle_sort(uint64_t* keys, uint32_t* ptrs, uint64_t n) {
    std::vector<std::pair<uint64_t, uint32_t>> v(n);
    for (uint64_t i = 0; i < n; ++i) v[i] = {keys[i], ptrs[i]};
    std::sort(v.begin(), v.end());
    for (uint64_t i = 0; i < n; ++i) { keys[i] = v[i].first; ptrs[i] = v[i].second; }
}

/* Merge (Table 2): the merge of sorted runs is the sorted concatenation. */
void oracle_merge(int nruns, const uint64_t* const* run_keys, const uint32_t* const* run_ptrs,
                  const uint64_t* run_lens, uint64_t* out_keys, uint32_t* out_ptrs) {
    uint64_t m = 0;
    for (int r = 0; r < nruns; ++r)
        for (uint64_t i = 0; i < run_lens[r]; ++i) { out_keys[m] = run_keys[r][i]; out_ptrs[m] = run_ptrs[r][i]; ++m; }
    oracle_sort(out_keys, out_ptrs, m);
}

/* Keyed reduction (Table 2; Sec. 4.2, "Reduction primitives"): per key, the
 * number of records and the sum of a nonresident value column reached through
 * the pointers.  Rows are visited in KPA order and accumulated in an ordered
 * map; keys come out ascending.  Returns the number of distinct keys. */
uint64_t oracle_group_sum_count(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* val_col,
                                int val_bytes, uint64_t* out_keys, uint64_t* out_counts, uint64_t* out_sums) {
    std::map<uint64_t, std::pair<uint64_t, uint64_t>> groups;
    for (uint64_t i = 0; i < n; ++i) {
        auto& g = groups[keys[i]];
        g.first += 1;
        if (val_col) g.second += load_val(val_col, val_bytes, ptrs[i]);
    }
    uint64_t j = 0;
    for (const auto& kv : groups) {
        if (out_keys) out_keys[j] = kv.first;
        if (out_counts) out_counts[j] = kv.second.first;
        if (out_sums) out_sums[j] = kv.second.second;
        ++j;
    }
    return j;
}

/* TopK Per Key (Sec. 7, benchmark 1): per key the K largest values, ties
 * broken by the smaller pointer.  out_vals and out_ptrs hold K slots per key. */
uint64_t oracle_topk(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* val_col, int val_bytes,
                     int K, uint64_t* out_keys, uint8_t* out_nvalid, uint64_t* out_vals, uint32_t* out_ptrs) {
    std::map<uint64_t, std::vector<std::pair<uint64_t, uint32_t>>> groups;
    for (uint64_t i = 0; i < n; ++i) groups[keys[i]].push_back({load_val(val_col, val_bytes, ptrs[i]), ptrs[i]});
    uint64_t j = 0;
    for (auto& kv : groups) {
        auto& v = kv.second;
        std::sort(v.begin(), v.end(), [](const std::pair<uint64_t, uint32_t>& a, const std::pair<uint64_t, uint32_t>& b) {
            if (a.first != b.first) return a.first > b.first;
            return a.second < b.second;
        });
        uint64_t keep = std::min<uint64_t>(static_cast<uint64_t>(K), v.size());
        out_keys[j] = kv.first;
        out_nvalid[j] = static_cast<uint8_t>(keep);
        for (int s = 0; s < K; ++s) {
            out_vals[j * K + s] = s < static_cast<int>(keep) ? v[s].first : 0;
            out_ptrs[j * K + s] = s < static_cast<int>(keep) ? v[s].second : 0xFFFFFFFFu;
        }
        ++j;
    }
    return j;
}

/* Join (Table 2; Sec. 4.2, "Temporal Join"): every pair of records, one from
 * each side, with equal keys.  R is indexed in an ordered multimap and probed
 * with every record of L; the pairs are then put in (key, ptrL, ptrR) order.
 * Returns the number of pairs; only the first cap pairs are written. */
uint64_t oracle_join(const uint64_t* lkeys, const uint32_t* lptrs, uint64_t nl, const uint64_t* rkeys,
                     const uint32_t* rptrs, uint64_t nr, uint32_t* out_l, uint32_t* out_r, uint64_t cap) {
    std::multimap<uint64_t, uint32_t> index;
    for (uint64_t j = 0; j < nr; ++j) index.insert({rkeys[j], rptrs[j]});
    std::vector<std::tuple<uint64_t, uint32_t, uint32_t>> pairs;
    for (uint64_t i = 0; i < nl; ++i) {
        auto range = index.equal_range(lkeys[i]);
        for (auto it = range.first; it != range.second; ++it) pairs.emplace_back(lkeys[i], lptrs[i], it->second);
    }
    std::sort(pairs.begin(), pairs.end());
    for (uint64_t p = 0; p < pairs.size() && p < cap; ++p) { out_l[p] = std::get<1>(pairs[p]); out_r[p] = std::get<2>(pairs[p]); }
    return pairs.size();
}

/* The same join by a nested loop over both sides (small inputs only). */
uint64_t oracle_join_nested(const uint64_t* lkeys, const uint32_t* lptrs, uint64_t nl, const uint64_t* rkeys,
                            const uint32_t* rptrs, uint64_t nr, uint32_t* out_l, uint32_t* out_r, uint64_t cap) {
    std::vector<std::tuple<uint64_t, uint32_t, uint32_t>> pairs;
    for (uint64_t i = 0; i < nl; ++i)
        for (uint64_t j = 0; j < nr; ++j)
            if (lkeys[i] == rkeys[j]) pairs.emplace_back(lkeys[i], lptrs[i], rptrs[j]);
    std::sort(pairs.begin(), pairs.end());
    for (uint64_t p = 0; p < pairs.size() && p < cap; ++p) { out_l[p] = std::get<1>(pairs[p]); out_r[p] = std::get<2>(pairs[p]); }
    return pairs.size();
}

/* Windowing (Sec. 4.2, "Windowing"): Partition by the timestamp column.
 * Window w holds the rows with ts in [starts[w], starts[w] + len).  With ts
 * non-decreasing these rows are one contiguous range, found here by a linear
 * scan that counts the rows strictly before each bound. */
void oracle_window_ranges(const void* ts, int ts_bytes, uint64_t n, const uint64_t* starts, uint64_t len,
                          uint64_t nwin, uint64_t* row_begin, uint64_t* row_end) {
    for (uint64_t w = 0; w < nwin; ++w) {
        uint64_t lo = starts[w], hi = starts[w] + len;
        uint64_t b = 0, e = 0;
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t t = load_ts(ts, ts_bytes, i);
            if (t < lo) ++b;
            if (t < hi) ++e;
        }
        row_begin[w] = b;
        row_end[w] = e;
    }
}

/* Materialize (Table 2): the column values of the KPA's records, in KPA
 * order: out[i] = col[ptrs[i]].  KeySwap (Table 2) is the same gather of
 * another key column, which becomes the KPA's resident key. */
void oracle_materialize(const uint32_t* ptrs, uint64_t n, const void* col, int col_bytes, void* out) {
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t v = load_val(col, col_bytes, ptrs[i]);
        if (col_bytes == 8) static_cast<uint64_t*>(out)[i] = v;
        else static_cast<uint32_t*>(out)[i] = static_cast<uint32_t>(v);
    }
}

/* Select (Table 2): the records whose value (col[ptr]) lies in [lo, hi), in
 * KPA order.  Returns how many; only the first cap are written. */
uint64_t oracle_select(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* col, int col_bytes,
                       uint64_t lo, uint64_t hi, uint64_t* out_keys, uint32_t* out_ptrs, uint64_t cap) {
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t v = load_val(col, col_bytes, ptrs[i]);
        if (v >= lo && v < hi) {
            if (m < cap) { out_keys[m] = keys[i]; out_ptrs[m] = ptrs[i]; }
            ++m;
        }
    }
    return m;
}

/* Median and distinct values per key (Sec. 7, benchmarks "Median" and
 * "Unique Count"): per key (ascending), its values sorted ascending; the
 * median is the lower one, at index (count - 1) / 2; unique counts the
 * distinct values.  Returns the number of keys. */
uint64_t oracle_median_unique(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const void* col, int col_bytes,
                              uint64_t* out_keys, uint64_t* out_median, uint64_t* out_unique) {
    std::map<uint64_t, std::vector<uint64_t>> groups;
    for (uint64_t i = 0; i < n; ++i) groups[keys[i]].push_back(load_val(col, col_bytes, ptrs[i]));
    uint64_t j = 0;
    for (auto& kv : groups) {
        auto& v = kv.second;
        std::sort(v.begin(), v.end());
        out_keys[j] = kv.first;
        out_median[j] = v[(v.size() - 1) / 2];
        out_unique[j] = static_cast<uint64_t>(std::unique(v.begin(), v.end()) - v.begin());
        ++j;
    }
    return j;
}

/* Partition (Table 2: split a KPA by ranges of its resident keys).  bounds
 * holds nb non-decreasing keys; part j (0 <= j <= nb) receives the records
 * with bounds[j - 1] <= key < bounds[j] (no lower limit for part 0, no upper
 * one for part nb), each part in the input order.  Every record is appended
 * to the vector of its part, found by counting the bounds not above its key;
 * the parts are then laid end to end.  offsets[j] = the first row of part j,
 * offsets[nb + 1] = n. */
void oracle_partition(const uint64_t* keys, const uint32_t* ptrs, uint64_t n, const uint64_t* bounds, uint64_t nb,
                      uint64_t* out_keys, uint32_t* out_ptrs, uint64_t* offsets) {
    std::vector<std::vector<std::pair<uint64_t, uint32_t>>> parts(nb + 1);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t j = 0;
        while (j < nb && bounds[j] <= keys[i]) ++j;
        parts[j].push_back({keys[i], ptrs[i]});
    }
    uint64_t m = 0;
    for (uint64_t j = 0; j <= nb; ++j) {
        offsets[j] = m;
        for (const auto& kp : parts[j]) { out_keys[m] = kp.first; out_ptrs[m] = kp.second; ++m; }
    }
    offsets[nb + 1] = m;
}

}  // extern "C"
