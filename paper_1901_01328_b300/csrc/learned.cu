// A4 Learned MSD partition sort.  The paper sorts KPAs with an in-core merge
// sort (Sec. 4.2, "Primitive Implementation"); this path instead derives MSD
// bucket boundaries from a small network fitted to the keys' CDF, so that
// one scatter by bucket (two or three digit passes over a short bucket id)
// leaves buckets small enough to sort in shared memory.
//
// Cells.  Key 0 is cell 0; a key k >= 1 with highest set bit m lies in cell
// 1 + 1024 m + (the 10 bits below bit m); the next 32 bits are its offset in
// the cell.  Cells with m <= 10 hold exactly one key value.
//
// Training (sbh_learned_train).  The sample is sorted; key values whose
// sample count stands for more than half a bucket are heavy and get one
// dedicated bucket each; the other samples form the training set: row r takes the
// sorted non-heavy sample (r * P) mod m', input x = feature(key) (exact in
// FP32), target = midpoint of the key's CDF step among those samples.  A
// 1-32-32-1 ReLU network is fitted by Adam on mean squared error; G CTAs
// each compute the gradient of a slice of every batch, meet at a grid
// barrier, each CTA sums one slice of the parameters over all partial
// gradients in a fixed order and applies Adam to it, and meet again.
//
// Partition (sbh_kpa_sort_learned).  F(c) = the prefix maximum of the
// clamped network output at each cell's lowest key; cell c spans
// y(c) = floor(F(c + 1) NB) - floor(F(c) NB) spread buckets plus two per
// heavy key in it, and its first bucket t(c) is floor(F(c) NB) plus two per
// heavy key in the cells before it.  Key k of cell c goes to bucket
//   t(c) + floor(offset(k) * y(c) / 2^32) + 2 * (heavy keys of c below k)
//        + (1 if k is heavy),
// so a heavy key has a bucket of its own (its neighbours' buckets differ by
// the parity of the heavy term).  Bucket ids are therefore non-decreasing in
// the key (integer arithmetic only), so a stable sort by bucket id followed
// by a sort inside each bucket sorts the KPA.  Buckets of one key are already
// in input order; buckets above the shared-memory capacity go to the plain
// radix sort.  Every step is stable, so rows of equal keys keep their input
// order, as in the plain sort.
#include <algorithm>
#include <vector>

#include "radix_core.cuh"

namespace sbh {
namespace {

constexpr int kH = 32;
constexpr int kNP = 4 * kH + kH * kH + 1;  // 1153
constexpr int oW1 = 0, oB1 = kH, oW2 = 2 * kH, oB2 = 2 * kH + kH * kH, oW3 = 3 * kH + kH * kH, oB3 = 4 * kH + kH * kH;
constexpr uint32_t kNCell = 1 + 64 * 1024;
constexpr uint32_t kMaxHeavy = SBH_LEARNED_MAX_HEAVY;
constexpr uint32_t kMaxBucketIds = 1u << 16;  // ids carried in 16 bits
constexpr uint32_t kHeavyDiv = 2;

struct Model {
    float params[kNP];
    uint32_t capacity;     // rows a bucket may hold to be sorted in shared memory
    uint32_t heavy_count;  // heavy keys (at most kMaxHeavy once trained)
    uint32_t m_train;      // rows of the training set
    uint32_t reserved[2];
    uint64_t heavy_keys[kMaxHeavy];  // ascending
};
static_assert(sizeof(Model) <= SBH_LEARNED_MODEL_BYTES, "model blob");
static_assert(offsetof(Model, heavy_keys) == 4 * (kNP + 5), "model layout");

// Index of key k in the model's heavy keys, or -1 (binary search).
__device__ __forceinline__ int heavy_index(const Model* __restrict__ model, uint64_t k) {
    uint32_t lo = 0, hi = min(model->heavy_count, kMaxHeavy);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (model->heavy_keys[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < min(model->heavy_count, kMaxHeavy) && model->heavy_keys[lo] == k) ? static_cast<int>(lo) : -1;
}

// ------------------------------------------------------------------ key features
__device__ __forceinline__ float key_feature(uint64_t k) {
    if (!k) return 0.f;
    const int m = 63 - __clzll(static_cast<long long>(k));
    const uint64_t top = k << (63 - m);
    const uint32_t f = static_cast<uint32_t>(top >> 46) & 0x1FFFFu;
    return (static_cast<float>(m) + static_cast<float>(f) * (1.0f / 131072.0f)) * (1.0f / 64.0f);
}

__device__ __forceinline__ uint32_t key_cell(uint64_t k, uint32_t* frac) {
    if (!k) {
        *frac = 0;
        return 0;
    }
    const int m = 63 - __clzll(static_cast<long long>(k));
    const uint64_t top = k << (63 - m);
    *frac = static_cast<uint32_t>((top << 11) >> 32);
    return 1u + 1024u * static_cast<uint32_t>(m) + static_cast<uint32_t>((top >> 53) & 1023u);
}

__host__ __device__ __forceinline__ bool cell_exact(uint32_t c) { return c == 0 || (c - 1) / 1024 <= 10; }

// feature of the lowest key of cell c (c == kNCell: the end of key space)
__device__ __forceinline__ float cell_x(uint32_t c) {
    if (c == 0) return 0.f;
    if (c >= kNCell) return 1.f;
    const uint32_t m = (c - 1) / 1024, b = (c - 1) % 1024;
    return (static_cast<float>(m) + static_cast<float>(b) * (1.0f / 1024.0f)) * (1.0f / 64.0f);
}

// ------------------------------------------------------------------ network
__device__ __forceinline__ float mlp_eval(const float* __restrict__ P, float x) {
    float h1[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) h1[i] = fmaxf(fmaf(P[oW1 + i], x, P[oB1 + i]), 0.f);
    float y = P[oB3];
#pragma unroll 4
    for (int o = 0; o < kH; ++o) {
        float a = P[oB2 + o];
#pragma unroll
        for (int i = 0; i < kH; ++i) a = fmaf(P[oW2 + o * kH + i], h1[i], a);
        y = fmaf(P[oW3 + o], fmaxf(a, 0.f), y);
    }
    return y;
}

constexpr int kGThreads = 1024;
constexpr int kMaxSlice = 256;
constexpr int kTrainCtas = 32;  // batch rows per CTA = batch / 32, in slices of at most kMaxSlice
constexpr int kBatchUnit = 128, kMaxBatch = 32768;  // the batch sizes the training takes
static_assert(kBatchUnit % kTrainCtas == 0, "whole rows per CTA");

struct GradSmem {
    float P[kNP];
    float W2T[kH * kH];  // W2 transposed: lanes that differ in the output unit read consecutive words
    float G[kNP];
    float X[kMaxSlice], T[kMaxSlice], DY[kMaxSlice];
    float A1[kMaxSlice][kH + 1];
    float A2[kMaxSlice][kH + 1];
    float D2[kMaxSlice][kH + 1];  // dL/da2
    float part[4][kNP];           // gradient sums over the rows s = k (mod 4), laid out like G
    float red[kGThreads / 32];
    float GA[kNP];           // training: the gradient over this CTA's rows (its slices summed)
    float AM[kNP], AV[kNP];  // training: Adam's moments (the same in every CTA)
};

// Gradient of sum_s (y_s - t_s)^2 / norm over the S rows in sm.X, sm.T into
// sm.G (and the sum of squared errors, returned to thread 0).  sm.P holds the
// parameters.  Every sum runs in a fixed order: a sum over rows keeps four
// partial sums (rows s = k mod 4, each in row order) combined as
// (k0 + k1) + (k2 + k3); a sum over units runs in unit order.  The three
// 32-wide products (second layer forward, its weight gradient and the
// gradient back to the first layer) take 4 x 4 register tiles, so each
// shared-memory load feeds four multiply-adds.  (2 x 2 tiles, which keep all
// 1024 threads busy at 128 rows, measured slower: the bench's training 0.65
// against 0.57 ms; so did splitting each 32-term sum between the two lanes
// of a pair, 0.58 ms with the weights' rows padded against bank conflicts.)
__device__ float slice_grad(GradSmem& sm, int S, float norm) {
    const int tid = threadIdx.x;
    const int stiles = (S + 3) / 4;  // groups of four rows
    for (int e = tid; e < kH * kH; e += kGThreads) sm.W2T[(e % kH) * kH + e / kH] = sm.P[oW2 + e];
    for (int e = tid; e < S * kH; e += kGThreads) {
        const int s = e / kH, i = e % kH;
        sm.A1[s][i] = fmaf(sm.P[oW1 + i], sm.X[s], sm.P[oB1 + i]);
    }
    __syncthreads();
    // a2[s][o] = b2[o] + sum_i W2[o][i] relu(a1[s][i]), rows s0..s0+3, units o0..o0+3
    for (int t = tid; t < stiles * (kH / 4); t += kGThreads) {
        const int s0 = (t / (kH / 4)) * 4, o0 = (t % (kH / 4)) * 4;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = sm.P[oB2 + o0 + c];
#pragma unroll 4
        for (int i = 0; i < kH; ++i) {
            float h[4], w[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) h[r] = fmaxf(sm.A1[s0 + r][i], 0.f);
#pragma unroll
            for (int c = 0; c < 4; ++c) w[c] = sm.W2T[i * kH + o0 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(w[c], h[r], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (s0 + r < S)
#pragma unroll
                for (int c = 0; c < 4; ++c) sm.A2[s0 + r][o0 + c] = acc[r][c];
    }
    __syncthreads();
    float sq = 0.f;
    for (int s = tid; s < S; s += kGThreads) {
        float y = sm.P[oB3];
#pragma unroll 8
        for (int o = 0; o < kH; ++o) y = fmaf(sm.P[oW3 + o], fmaxf(sm.A2[s][o], 0.f), y);
        const float r = y - sm.T[s];
        sm.DY[s] = 2.f * r / norm;
        sq += r * r;
    }
    __syncthreads();
    // w3, b3 partial sums (threads 0..131); dL/da2 (all threads)
    if (tid < 4 * (kH + 1)) {
        const int k = tid / (kH + 1), o = tid % (kH + 1);
        float g = 0.f;
        if (o < kH) {
            for (int s = k; s < S; s += 4) g = fmaf(sm.DY[s], fmaxf(sm.A2[s][o], 0.f), g);
            sm.part[k][oW3 + o] = g;
        } else {
            for (int s = k; s < S; s += 4) g += sm.DY[s];
            sm.part[k][oB3] = g;
        }
    }
    for (int e = tid; e < S * kH; e += kGThreads) {
        const int s = e / kH, o = e % kH;
        sm.D2[s][o] = sm.A2[s][o] > 0.f ? sm.DY[s] * sm.P[oW3 + o] : 0.f;
    }
    __syncthreads();
    // W2 partial sums in 4 x 4 tiles of (o, i) (threads 0..255), b2 partial
    // sums (threads 256..383); w3, b3 combined (threads 384..416)
    if (tid < 4 * 64) {
        const int k = tid / 64, tile = tid % 64;
        const int o0 = (tile / 8) * 4, i0 = (tile % 8) * 4;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
        for (int s = k; s < S; s += 4) {
            float d[4], h[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) d[r] = sm.D2[s][o0 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) h[c] = fmaxf(sm.A1[s][i0 + c], 0.f);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(d[r], h[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) sm.part[k][oW2 + (o0 + r) * kH + i0 + c] = acc[r][c];
    } else if (tid < 4 * 64 + 4 * kH) {
        const int k = (tid - 4 * 64) / kH, o = (tid - 4 * 64) % kH;
        float g = 0.f;
        for (int s = k; s < S; s += 4) g += sm.D2[s][o];
        sm.part[k][oB2 + o] = g;
    } else if (tid < 4 * 64 + 4 * kH + kH + 1) {
        const int j = tid - (4 * 64 + 4 * kH) + oW3;  // oW3 .. oB3
        sm.G[j] = (sm.part[0][j] + sm.part[1][j]) + (sm.part[2][j] + sm.part[3][j]);
    }
    __syncthreads();
    // W2, b2 combined; dL/da1 = (sum_o dL/da2[s][o] W2[o][i]) where a1 > 0,
    // in 4 x 4 tiles of (s, i), written over A1 (each entry by its own thread;
    // the reads of A1 for W2 ended at the barrier above)
    for (int j = oW2 + tid; j < oW3; j += kGThreads)
        sm.G[j] = (sm.part[0][j] + sm.part[1][j]) + (sm.part[2][j] + sm.part[3][j]);
    for (int t = tid; t < stiles * (kH / 4); t += kGThreads) {
        const int s0 = (t / (kH / 4)) * 4, i0 = (t % (kH / 4)) * 4;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 4
        for (int o = 0; o < kH; ++o) {
            float d[4], w[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) d[r] = sm.D2[s0 + r][o];
#pragma unroll
            for (int c = 0; c < 4; ++c) w[c] = sm.P[oW2 + o * kH + i0 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(d[r], w[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (s0 + r < S)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    sm.A1[s0 + r][i0 + c] = sm.A1[s0 + r][i0 + c] > 0.f ? acc[r][c] : 0.f;
    }
    __syncthreads();
    // W1, b1 partial sums (threads 0..255)
    if (tid < 4 * 2 * kH) {
        const int k = tid / (2 * kH), i = tid % (2 * kH);
        float g = 0.f;
        if (i < kH) {
            for (int s = k; s < S; s += 4) g = fmaf(sm.A1[s][i], sm.X[s], g);
            sm.part[k][oW1 + i] = g;
        } else {
            for (int s = k; s < S; s += 4) g += sm.A1[s][i - kH];
            sm.part[k][oB1 + i - kH] = g;
        }
    }
    // sum of squared errors: warp shuffles, then warp totals in order
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if ((tid & 31) == 0) sm.red[tid / 32] = sq;
    __syncthreads();
    if (tid < 2 * kH) sm.G[tid] = (sm.part[0][tid] + sm.part[1][tid]) + (sm.part[2][tid] + sm.part[3][tid]);
    float tot = 0.f;
    if (tid == 0)
        for (int w = 0; w < kGThreads / 32; ++w) tot += sm.red[w];
    return tot;
}

// ---- forward and gradient entry kernels (tests and tools)
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* __restrict__ params, const float* __restrict__ x,
                                                          uint64_t m, float* __restrict__ y) {
    __shared__ float P[kNP];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < m) y[i] = mlp_eval(P, x[i]);
}

__global__ void __launch_bounds__(kGThreads) mlp_grad_partial_kernel(const float* __restrict__ params,
                                                                     const float* __restrict__ x,
                                                                     const float* __restrict__ t, uint64_t m,
                                                                     float* __restrict__ partial,
                                                                     float* __restrict__ partial_sq) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GradSmem& sm = *reinterpret_cast<GradSmem*>(smem_raw);
    for (int i = threadIdx.x; i < kNP; i += kGThreads) sm.P[i] = params[i];
    const uint64_t lo = blockIdx.x * (uint64_t)kMaxSlice;
    const int S = (int)min_u64(kMaxSlice, m - lo);
    for (int s = threadIdx.x; s < S; s += kGThreads) {
        sm.X[s] = x[lo + s];
        sm.T[s] = t[lo + s];
    }
    __syncthreads();
    const float sq = slice_grad(sm, S, static_cast<float>(m));
    __syncthreads();
    for (int i = threadIdx.x; i < kNP; i += kGThreads) partial[blockIdx.x * (size_t)kNP + i] = sm.G[i];
    if (threadIdx.x == 0) partial_sq[blockIdx.x] = sq;
}

__global__ void mlp_grad_sum_kernel(const float* __restrict__ partial, const float* __restrict__ partial_sq,
                                    uint32_t nparts, uint64_t m, float* __restrict__ grad, float* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNP) {
        float g = 0.f;
        for (uint32_t c = 0; c < nparts; ++c) g += partial[c * (size_t)kNP + i];
        grad[i] = g;
    }
    if (i == 0 && loss) {
        float l = 0.f;
        for (uint32_t c = 0; c < nparts; ++c) l += partial_sq[c];
        *loss = l / static_cast<float>(m);
    }
}

// ------------------------------------------------------------------ training data
struct TrainScratch {
    uint64_t* s_keys;    // sorted sample (m)
    uint32_t* s_ptrs;    // the sort's pointers (not used)
    uint64_t* nh;        // non-heavy sorted samples (m)
    uint32_t* flags;     // m + 1 (compaction)
    uint64_t* block_sums;
    float* X;
    float* T;
    float* partial;      // 2 x G x kNP (by step parity)
    float* partial_sq;   // 2 x G
    float* params;       // initial, then trained parameters
    uint32_t* bar;       // grid barrier: count, generation
    uint32_t* m_train;
    void* sort_scratch;
    size_t total;
};

constexpr int kCompactTile = 1024;

TrainScratch train_carve(void* base, uint64_t m) {
    Carver c(base);
    TrainScratch t;
    t.s_keys = c.take<uint64_t>(m);
    t.s_ptrs = c.take<uint32_t>(m);
    t.nh = c.take<uint64_t>(m);
    t.flags = c.take<uint32_t>(m + 1);
    t.block_sums = c.take<uint64_t>((m + kCompactTile - 1) / kCompactTile + 1);
    t.X = c.take<float>(m);
    t.T = c.take<float>(m);
    t.partial = c.take<float>(2 * kTrainCtas * (size_t)kNP);
    t.partial_sq = c.take<float>(2 * kTrainCtas);
    t.params = c.take<float>(kNP);
    t.bar = c.take<uint32_t>(2);
    t.m_train = c.take<uint32_t>(1);
    t.sort_scratch = c.take<char>(sort_carve(nullptr, m).total);
    t.total = c.bytes();
    return t;
}

// Heavy keys from the sorted sample: a run of count samples is heavy when
// count * n_rows > (capacity / kHeavyDiv) * m, i.e. count >= c_min =
// floor((capacity / kHeavyDiv) * m / n_rows) + 1, so the first sample of a
// run compares itself with the sample c_min - 1 places on.  A key of more
// than half a bucket gets a bucket of its own (an eighth measured the same:
// fewer rows left to sort, but more ids that take the heavy-cell path).
struct HeavyRunStart {
    const uint64_t* srt;
    uint64_t m, c_min;
    __device__ __forceinline__ bool operator()(uint64_t i) const {
        const uint64_t key = srt[i];
        if (i > 0 && srt[i - 1] == key) return false;
        return i + c_min - 1 < m && srt[i + c_min - 1] == key;
    }
};

// Samples that are not heavy keys (the training set's rows).
struct NotHeavy {
    const uint64_t* srt;
    const Model* model;
    __device__ __forceinline__ bool operator()(uint64_t i) const { return heavy_index(model, srt[i]) < 0; }
};

// Ordered compaction of the sorted samples that satisfy a predicate: per-tile
// counts, one-CTA scan, scatter (the first cap of them are written).
template <typename Pred>
__global__ void __launch_bounds__(kCompactTile) compact_count_kernel(uint64_t m, Pred pred,
                                                                     uint64_t* __restrict__ block_sums) {
    __shared__ uint32_t wsum[kCompactTile / 32];
    const uint64_t i = blockIdx.x * (uint64_t)kCompactTile + threadIdx.x;
    const uint32_t keep = i < m && pred(i);
    const uint32_t b = __popc(__ballot_sync(0xffffffffu, keep));
    if (lane_id() == 0) wsum[threadIdx.x / 32] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kCompactTile / 32; ++w) t += wsum[w];
        block_sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) scan_u64_kernel(uint64_t* __restrict__ v, uint32_t nb,
                                                        uint32_t* __restrict__ total32) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nb; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        const uint64_t x0 = i < nb ? v[i] : 0;
        uint64_t x = x0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (uint32_t)o) x += y;
        }
        if (lane_id() == 31) warp_tot[threadIdx.x / 32] = x;
        __syncthreads();
        uint64_t before = carry;
        for (uint32_t w = 0; w < threadIdx.x / 32; ++w) before += warp_tot[w];
        if (i < nb) v[i] = before + x - x0;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total32 = static_cast<uint32_t>(carry);
}

template <typename Pred>
__global__ void __launch_bounds__(kCompactTile) compact_scatter_kernel(const uint64_t* __restrict__ srt, uint64_t m,
                                                                       Pred pred,
                                                                       const uint64_t* __restrict__ block_off,
                                                                       uint64_t* __restrict__ out, uint64_t cap) {
    __shared__ uint32_t wsum[kCompactTile / 32];
    const uint64_t i = blockIdx.x * (uint64_t)kCompactTile + threadIdx.x;
    const uint32_t keep = i < m && pred(i);
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane_id() == 0) wsum[threadIdx.x / 32] = __popc(bal);
    __syncthreads();
    uint64_t off = block_off[blockIdx.x];
    for (uint32_t w = 0; w < threadIdx.x / 32; ++w) off += wsum[w];
    off += __popc(bal & lanemask_lt());
    if (keep && off < cap) out[off] = srt[i];
}

__device__ __forceinline__ uint32_t gcd_u32(uint32_t a, uint32_t b) {
    while (b) {
        const uint32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Training rows: row r takes sorted non-heavy sample (r * P) mod m'.
__global__ void trainset_kernel(const uint64_t* __restrict__ nh, const uint32_t* __restrict__ m_train,
                                float* __restrict__ X, float* __restrict__ T) {
    __shared__ uint32_t sP;
    const uint32_t mt = *m_train;
    if (mt == 0) return;
    if (threadIdx.x == 0) {
        uint32_t P = static_cast<uint32_t>(2654435761ull % mt);
        while (gcd_u32(P, mt) != 1) ++P;
        sP = P;
    }
    __syncthreads();
    const uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (r >= mt) return;
    const uint64_t j = (r * (uint64_t)sP) % mt;
    const uint64_t key = nh[j];
    // the key's run [lt, le) in the sorted samples: usually j alone, else
    // found by binary search on the side where it continues
    uint64_t lt = j, le = j + 1;
    if (j > 0 && nh[j - 1] == key) {
        uint64_t lo = 0, hi = j;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) / 2;
            if (nh[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        lt = lo;
    }
    if (j + 1 < mt && nh[j + 1] == key) {
        uint64_t lo = j + 1, hi = mt;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) / 2;
            if (nh[mid] <= key) lo = mid + 1;
            else hi = mid;
        }
        le = lo;
    }
    X[r] = key_feature(key);
    T[r] = static_cast<float>(lt + le) / (2.0f * static_cast<float>(mt));
}

// Start from the piecewise-linear interpolation of the training set's CDF at
// 33 quantiles (when no initial weights are given).  Knot i is the sorted
// non-heavy sample j = floor(i (m' - 1) / 32): x = feature(key), F = its CDF
// target; a knot with the x of the previous kept knot merges into it (taking
// the later F).  Unit u kinks at kept knot u (W1 = 1, b1 = -x_u), the second
// layer passes it on (W2 = I), w3_u is the change of slope at knot u and b3
// the first F, so the output passes through the kept knots.  One CTA.
__global__ void quantile_init_kernel(const uint64_t* __restrict__ nh, const uint32_t* __restrict__ m_train,
                                     float* __restrict__ params) {
    __shared__ float qx[kH + 1], qf[kH + 1];
    const uint32_t mt = *m_train;
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) params[i] = 0.f;
    if (threadIdx.x <= kH && mt > 0) {
        const uint32_t j = static_cast<uint32_t>((static_cast<uint64_t>(threadIdx.x) * (mt - 1)) / kH);
        const uint64_t key = nh[j];
        uint32_t lo = 0, hi = mt;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            if (nh[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        const uint32_t lt = lo;
        hi = mt;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            if (nh[mid] <= key) lo = mid + 1;
            else hi = mid;
        }
        qx[threadIdx.x] = key_feature(key);
        qf[threadIdx.x] = static_cast<float>(lt + lo) / (2.0f * static_cast<float>(mt));
    }
    __syncthreads();
    if (threadIdx.x != 0 || mt == 0) return;
    float kx[kH + 1], kf[kH + 1];
    int k = 0;
    for (int i = 0; i <= kH; ++i) {
        if (k > 0 && qx[i] <= kx[k - 1]) {
            kf[k - 1] = qf[i];
        } else {
            kx[k] = qx[i];
            kf[k] = qf[i];
            ++k;
        }
    }
    for (int u = 0; u < kH; ++u) params[oW2 + u * kH + u] = 1.f;
    float prev = 0.f;
    for (int u = 0; u + 1 < k; ++u) {
        const float slope = (kf[u + 1] - kf[u]) / (kx[u + 1] - kx[u]);
        params[oW1 + u] = 1.f;
        params[oB1 + u] = -kx[u];
        params[oW3 + u] = slope - prev;
        prev = slope;
    }
    params[oB3] = kf[0];
}

// ------------------------------------------------------------------ training
// Bounded grid barrier for the co-resident CTAs of a cooperative launch.
__device__ bool grid_barrier(uint32_t* bar, uint32_t nblocks, uint32_t spin_limit, uint32_t* status) {
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        volatile uint32_t* gen = bar + 1;
        const uint32_t g = *gen;
        __threadfence();
        const uint32_t arrived = atomicAdd(bar, 1u) + 1;
        if (arrived == nblocks) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            uint32_t polls = 0;
            while (*gen == g) {
                if (wait_expired(polls, spin_limit, status)) {
                    ok = false;
                    break;
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
    return ok;
}

struct TrainArgs {
    const float* X;
    const float* T;
    const uint32_t* m_train;
    float* params;      // initial weights in, trained weights out
    float* partial;     // 2 x G x kNP: each CTA's gradient, by step parity
    float* partial_sq;  // 2 x G
    uint32_t* bar;
    float* losses;   // nullable, one per step
    int steps;
    int batch;
    float lr;
    uint32_t spin_limit;
    uint32_t* status;
};

// Adam on the batch gradient with one grid barrier a step: each CTA takes
// batch / G rows (slices of at most kMaxSlice), writes its gradient to the
// buffer of the step's parity, and after the barrier every CTA sums the G
// gradients in CTA order and applies the same Adam update to its own copy of
// the parameters in shared memory, so the copies stay identical and no second
// barrier is needed.  A CTA writes the other parity's buffer next step only
// after every CTA has reached this step's barrier, that is, after all of them
// have read the previous step's gradients.  (128 CTAs of 32 rows, each
// updating ten parameters between two grid barriers a step, took 0.60 ms for
// the bench's 40 steps of 4096 rows; one cluster of 16 CTAs of 256 rows,
// summing through distributed shared memory, 0.66 ms.)
__global__ void __launch_bounds__(kGThreads) train_kernel(TrainArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GradSmem& sm = *reinterpret_cast<GradSmem*>(smem_raw);
    const uint32_t mt = *a.m_train;
    const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
    const int S = a.batch / G;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float b1t = 1.f, b2t = 1.f;
    if (mt == 0) return;
    for (int i = tid; i < kNP; i += kGThreads) {
        sm.P[i] = a.params[i];
        sm.AM[i] = 0.f;
        sm.AV[i] = 0.f;
    }
    for (int step = 0; step < a.steps; ++step) {
        const int par = step & 1;
        float sq = 0.f;
        for (int s0 = 0; s0 < S; s0 += kMaxSlice) {
            const int ns = min(kMaxSlice, S - s0);
            __syncthreads();  // the previous slice (or step) is done with X, T, G and P
            for (int s = tid; s < ns; s += kGThreads) {
                const uint64_t row = ((uint64_t)step * a.batch + (uint64_t)c * S + s0 + s) % mt;
                sm.X[s] = a.X[row];
                sm.T[s] = a.T[row];
            }
            __syncthreads();
            sq += slice_grad(sm, ns, static_cast<float>(a.batch));
            __syncthreads();
            for (int i = tid; i < kNP; i += kGThreads) sm.GA[i] = s0 ? sm.GA[i] + sm.G[i] : sm.G[i];
        }
        float* part = a.partial + (size_t)par * G * kNP;
        for (int i = tid; i < kNP; i += kGThreads) part[(size_t)c * kNP + i] = sm.GA[i];
        if (tid == 0) a.partial_sq[par * G + c] = sq;
        __threadfence();
        if (!grid_barrier(a.bar, G, a.spin_limit, a.status)) return;
        b1t *= b1;
        b2t *= b2;
        for (int i = tid; i < kNP; i += kGThreads) {
            float g = 0.f;
            for (int q = 0; q < G; ++q) g += part[(size_t)q * kNP + i];
            const float mi = b1 * sm.AM[i] + (1.f - b1) * g;
            const float vi = b2 * sm.AV[i] + (1.f - b2) * g * g;
            sm.AM[i] = mi;
            sm.AV[i] = vi;
            const float mhat = mi / (1.f - b1t), vhat = vi / (1.f - b2t);
            sm.P[i] -= a.lr * mhat / (sqrtf(vhat) + eps);
        }
        if (c == 0 && tid == 0 && a.losses) {
            float l = 0.f;
            for (int q = 0; q < G; ++q) l += a.partial_sq[par * G + q];
            a.losses[step] = l / static_cast<float>(a.batch);
        }
    }
    __syncthreads();
    if (c == 0)
        for (int i = tid; i < kNP; i += kGThreads) a.params[i] = sm.P[i];
}

__global__ void finish_model_kernel(const float* __restrict__ params, const uint32_t* __restrict__ m_train,
                                    uint32_t capacity, Model* __restrict__ model) {
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) model->params[i] = params[i];
    if (threadIdx.x == 0) {
        model->capacity = capacity;
        model->m_train = *m_train;
        model->heavy_count = min(model->heavy_count, kMaxHeavy);
    }
}

// ------------------------------------------------------------------ partition
// Bucket id of a key (see the file comment).
// One 8-byte entry per cell, so an id mostly costs a single table load:
// x = the cell's first bucket id, y = its number of spread buckets; a cell
// holding heavy keys has y = kHeavyCell and x = the index of its first heavy
// key, under which hcells keeps the cell's HeavyCell entry.  An exact cell
// (one key value) that is heavy
// has y = kHeavyExact: its key's bucket is x + 1.
constexpr uint32_t kHeavyCell = 0xFFFFFFFFu;
constexpr uint32_t kHeavyExact = 0xFFFFFFFEu;

// A cell holding heavy keys: first bucket id, spread buckets, heavy keys in
// the cell, and the first two of them (one 32-byte sector: most such cells
// hold one or two, and then the id needs no load of the heavy-key list; the
// id upsweep for 256M hashed keys, whose heavy keys share cells with most
// rows, 1.28 to 1.15 ms, for the mixed keys 0.645 to 0.630 ms).
struct HeavyCell {
    uint32_t t, y, hv, pad;
    uint64_t k0, k1;
};

// The id of key k (offset f) in a cell holding heavy keys.
__device__ __forceinline__ uint32_t heavy_cell_id(const HeavyCell* __restrict__ hcells,
                                                  const uint64_t* __restrict__ hkeys, uint32_t idx, uint32_t f,
                                                  uint64_t k) {
    const uint4 h = __ldg(reinterpret_cast<const uint4*>(hcells + idx));
    const ulonglong2 hk2 = __ldg(reinterpret_cast<const ulonglong2*>(hcells + idx) + 1);
    uint32_t id = h.x + static_cast<uint32_t>((static_cast<uint64_t>(f) * h.y) >> 32);
    id += hk2.x < k ? 2u : (hk2.x == k ? 1u : 0u);
    if (h.z > 1) id += hk2.y < k ? 2u : (hk2.y == k ? 1u : 0u);
#pragma unroll 4
    for (uint32_t j = 2; j < h.z; ++j) {  // no early exit: the loads are independent
        const uint64_t hk = hkeys[idx + j];
        id += hk < k ? 2u : (hk == k ? 1u : 0u);
    }
    return id;
}

struct BucketValue {
    const uint2* cells;      // kNCell + 1 entries
    const HeavyCell* hcells;  // by first heavy key index
    const uint64_t* hkeys;   // the model's heavy keys
    __device__ __forceinline__ uint64_t operator()(uint64_t k) const {
        uint32_t f;
        const uint32_t c = key_cell(k, &f);
        const uint2 e = __ldg(cells + c);
        if (e.y >= kHeavyExact) return e.y == kHeavyExact ? e.x + 1 : heavy_cell_id(hcells, hkeys, e.x, f, k);
        return e.x + static_cast<uint32_t>((static_cast<uint64_t>(f) * e.y) >> 32);
    }
};

// The same ids from a 4-byte entry per cell (half the table, so more of it
// stays in L1), usable when every id is below 2^16: first id (or first heavy
// key index) in the low 16 bits, spread buckets (at most 2^16 - 2 then) or
// kHeavyCell16 / kHeavyExact16 in the high.  (A 2-byte first-id table read
// after a bit of a heavy-cell bitmap, a quarter of the 8-byte table's size,
// measured slower: the id upsweep for 256M mixed keys 0.90 against 0.65 ms,
// the bitmap load lengthening each lookup's chain of dependent loads.)
constexpr uint32_t kHeavyCell16 = 0xFFFFu;
constexpr uint32_t kHeavyExact16 = 0xFFFEu;

struct BucketValue16 {
    const uint32_t* cells;   // kNCell + 1 entries
    const HeavyCell* hcells;
    const uint64_t* hkeys;
    __device__ __forceinline__ uint64_t operator()(uint64_t k) const {
        uint32_t f;
        const uint32_t c = key_cell(k, &f);
        const uint32_t e = __ldg(cells + c);
        const uint32_t x = e & 0xFFFFu, y = e >> 16;
        if (y >= kHeavyExact16) return y == kHeavyExact16 ? x + 1 : heavy_cell_id(hcells, hkeys, x, f, k);
        return x + static_cast<uint32_t>((static_cast<uint64_t>(f) * y) >> 32);
    }
};

// The partition's spread-bucket count nb and the number of heavy keys that
// keep a bucket of their own, decided on the device from the model, so that
// the call needs no host synchronisation.  nb_n is about two buckets per
// capacity of rows.  With carry (ids travel in 16 bits), every id must stay
// below 2^16: up to a quarter fewer spread buckets are accepted for it, and
// if the heavy keys still do not fit, only the smallest of them keep their
// own bucket (the others are spread like any other key).  plan[0] = heavy
// keys used, plan[1] = nb.
__global__ void learned_plan_kernel(const Model* __restrict__ model, uint32_t nb_n, int carry,
                                    uint32_t* __restrict__ plan) {
    if (threadIdx.x != 0) return;
    uint32_t h = min(model->heavy_count, kMaxHeavy);
    uint32_t nb = nb_n;
    if (carry) {
        const uint32_t lo = nb_n - nb_n / 4;  // fewest spread buckets accepted (the host checked lo <= 65533)
        h = min(h, (kMaxBucketIds - 2u - lo) / 2u);
        nb = min(min(nb_n, kMaxBucketIds - 2u - 2u * h), kMaxBucketIds - 3u);
    }
    plan[0] = h;
    plan[1] = nb;
}

// Heavy keys per cell: their number and the index of the first (cell_hc
// zeroed, cell_hidx filled with 0xFF bytes beforehand), for the first
// *h_used heavy keys of the model.
__global__ void heavy_cells_kernel(const Model* __restrict__ model, const uint32_t* __restrict__ h_used,
                                   uint32_t* __restrict__ cell_hc, uint32_t* __restrict__ cell_hidx) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *h_used) return;
    uint32_t f;
    const uint32_t c = key_cell(model->heavy_keys[i], &f);
    atomicAdd(&cell_hc[c], 1u);
    atomicMin(&cell_hidx[c], i);
}

// The cell table is built over blocks of 1024 cells in two launches:
// cell_cdf writes F and each block's maximum of F and number of heavy keys;
// cell_table combines the blocks before its own and scans its block.
constexpr int kTblThreads = 1024;
constexpr uint32_t kTblBlocks = (kNCell + 1 + kTblThreads - 1) / kTblThreads;

__global__ void __launch_bounds__(kTblThreads) cell_cdf_kernel(const Model* __restrict__ model, float* __restrict__ F,
                                                               const uint32_t* __restrict__ cell_hc,
                                                               float* __restrict__ bmax,
                                                               uint32_t* __restrict__ bheavy) {
    __shared__ float P[kNP];
    __shared__ float wm[32];
    __shared__ uint32_t wc[32];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) P[i] = model->params[i];
    __syncthreads();
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x, lane = lane_id(), warp = threadIdx.x / 32;
    float f = 0.f;
    uint32_t h = 0;
    if (c <= kNCell) {
        f = fminf(fmaxf(mlp_eval(P, cell_x(c)), 0.f), 1.f);
        F[c] = f;
        h = c < kNCell ? cell_hc[c] : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        f = fmaxf(f, __shfl_xor_sync(0xffffffffu, f, o));
        h += __shfl_xor_sync(0xffffffffu, h, o);
    }
    if (lane == 0) {
        wm[warp] = f;
        wc[warp] = h;
    }
    __syncthreads();
    if (warp == 0) {
        f = wm[lane];
        h = wc[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f = fmaxf(f, __shfl_xor_sync(0xffffffffu, f, o));
            h += __shfl_xor_sync(0xffffffffu, h, o);
        }
        if (lane == 0) {
            bmax[blockIdx.x] = f;
            bheavy[blockIdx.x] = h;
        }
    }
}

// Cell c's first bucket id is t(c) = floor(max(F[0..c]) * nb) + 2 * (heavy
// keys in the cells before c); each heavy key's own bucket is marked in the
// bitmap of heavy buckets; nbid receives t(kNCell) + 1, the bound on bucket
// ids.
__global__ void __launch_bounds__(kTblThreads) cell_table_kernel(const Model* __restrict__ model,
                                                                 const float* __restrict__ F,
                                                                 const uint32_t* __restrict__ cell_hc,
                                                                 const uint32_t* __restrict__ cell_hidx,
                                                                 HeavyCell* __restrict__ hcells,
                                                                 const float* __restrict__ bmax,
                                                                 const uint32_t* __restrict__ bheavy,
                                                                 const uint32_t* __restrict__ nb_p,
                                                                 uint2* __restrict__ cells,
                                                                 uint32_t* __restrict__ cells16,
                                                                 uint32_t* __restrict__ heavy_bucket_bits,
                                                                 uint32_t* __restrict__ nbid) {
    __shared__ float wm[32];
    __shared__ uint32_t wc[32];
    __shared__ float pre_m;
    __shared__ uint32_t pre_h;
    const uint32_t blk = blockIdx.x, c = blk * kTblThreads + threadIdx.x, lane = lane_id(), warp = threadIdx.x / 32;
    if (warp == 0) {  // the blocks before this one
        float m = 0.f;
        uint32_t h = 0;
        for (uint32_t j = lane; j < blk; j += 32) {
            m = fmaxf(m, bmax[j]);
            h += bheavy[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            h += __shfl_xor_sync(0xffffffffu, h, o);
        }
        if (lane == 0) {
            pre_m = m;
            pre_h = h;
        }
    }
    const float f = c <= kNCell ? F[c] : 0.f;
    const uint32_t hv = c < kNCell ? cell_hc[c] : 0u;  // heavy keys in this cell
    float m = f;
    uint32_t h = hv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float ym = __shfl_up_sync(0xffffffffu, m, o);
        const uint32_t yh = __shfl_up_sync(0xffffffffu, h, o);
        if (lane >= (uint32_t)o) {
            m = fmaxf(m, ym);
            h += yh;
        }
    }
    if (lane == 31) {
        wm[warp] = m;
        wc[warp] = h;
    }
    __syncthreads();
    float bm = pre_m;
    uint32_t bh = pre_h;
    for (uint32_t w = 0; w < warp; ++w) {
        bm = fmaxf(bm, wm[w]);
        bh += wc[w];
    }
    const float run_max = fmaxf(bm, m);  // max of F[0..c]
    const uint32_t heavy_incl = bh + h;  // heavy keys in the cells [0, c]
    const float fnb = static_cast<float>(*nb_p);
    const uint32_t t = static_cast<uint32_t>(floorf(run_max * fnb)) + 2u * (heavy_incl - hv);
    // the next cell's first id (the same arithmetic as its own thread's)
    float f_next = __shfl_down_sync(0xffffffffu, f, 1);
    if (lane == 31) f_next = c + 1 <= kNCell ? F[c + 1] : 0.f;
    const uint32_t t_next = static_cast<uint32_t>(floorf(fmaxf(run_max, f_next) * fnb)) + 2u * heavy_incl;
    if (c > kNCell) return;
    if (c == kNCell) *nbid = t + 1;
    const uint32_t y = c == kNCell ? 0u : t_next - t - 2u * hv;  // spread buckets
    uint2 e;
    if (hv && cell_exact(c)) {  // one key value, heavy: bucket t + 1
        e = make_uint2(t, kHeavyExact);
        atomicOr(&heavy_bucket_bits[(t + 1) >> 5], 1u << ((t + 1) & 31));
    } else if (hv) {
        const uint32_t idx = cell_hidx[c];
        hcells[idx] = HeavyCell{t, y, hv, 0u, model->heavy_keys[idx], hv > 1 ? model->heavy_keys[idx + 1] : 0ull};
        e = make_uint2(idx, kHeavyCell);
        for (uint32_t j = 0; j < hv; ++j) {  // the heavy keys' own buckets
            uint32_t fh;
            key_cell(model->heavy_keys[idx + j], &fh);
            const uint32_t id = t + static_cast<uint32_t>((static_cast<uint64_t>(fh) * y) >> 32) + 2u * j + 1u;
            atomicOr(&heavy_bucket_bits[id >> 5], 1u << (id & 31));
        }
    } else {
        e = make_uint2(t, y);
    }
    cells[c] = e;
    // meaningful only when every id is below 2^16 (the carried-id path,
    // where spread counts stay below kHeavyExact16)
    const uint32_t y16 = e.y == kHeavyCell ? kHeavyCell16 : (e.y == kHeavyExact ? kHeavyExact16 : (e.y & 0xFFFFu));
    cells16[c] = (e.x & 0xFFFFu) | (y16 << 16);
}

// bstart[b] = first row whose bucket id is >= b, for b in [0, nbid].  Each
// row's id is computed once; lane 0 also computes the id of the row before.
__global__ void __launch_bounds__(256) bucket_bounds_kernel(const uint64_t* __restrict__ keys, uint32_t n,
                                                            BucketValue fn, const uint32_t* __restrict__ nbid_p,
                                                            uint32_t* __restrict__ bstart) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nbid = *nbid_p;
    const int64_t id = i < n ? static_cast<int64_t>(fn(ld_stream(keys + i))) : 0;
    int64_t prev = __shfl_up_sync(0xffffffffu, id, 1);
    if (lane_id() == 0) prev = (i > 0 && i <= n) ? static_cast<int64_t>(fn(keys[i - 1])) : -1;
    if (i >= n) return;
    for (int64_t b = prev + 1; b <= id; ++b) bstart[b] = i;
    if (i == n - 1)
        for (uint32_t b = static_cast<uint32_t>(id) + 1; b <= nbid; ++b) bstart[b] = n;
}

// In-shared-memory sort of each bucket of at most kCap rows.
constexpr uint32_t kCap = SBH_LEARNED_CAPACITY;
constexpr int kBThreads = 1024;
constexpr int kBWarps = kBThreads / 32;
static_assert(kBWarps == 32, "the bucket sort scans its warps' totals one per lane");
constexpr int kBIpt = kCap / kBThreads;
constexpr int kBGroups = kBThreads / 128;  // warp groups of the radix passes' count scan
constexpr int kBWpg = kBWarps / kBGroups;

constexpr int kFineBits = 12;
constexpr int kFineBins = 1 << kFineBits;
constexpr int kFinePer = kFineBins / kBThreads;  // bins scanned by each thread
constexpr uint32_t kFineMaxBin = 32;             // larger sub-buckets take the radix passes
constexpr int kWideBits = 40;  // ... unless the key range is wider: then a group sort and ranks
// Consecutive buckets are sorted together as one run of at most kCap rows
// (their key ranges are consecutive, so sorting the run sorts each bucket);
// a heavy bucket, or one of more than kCap rows, is a run of its own.
constexpr uint32_t kRunHeavy = 1u << 31, kRunEnd = kRunHeavy - 1;
constexpr int kGroupSubBits = 4;  // a big fine bin splits into 2^kGroupSubBits groups
constexpr int kGroupPasses = (kFineBits + kGroupSubBits + kRadixBits - 1) / kRadixBits;

struct BucketSmem {
    uint64_t keys[2][kCap];
    uint32_t ptrs[2][kCap];
    union {
        uint32_t bins[kFineBins];                   // counting placement by the top bits of key - kmin
        uint32_t whist2[kBWarps][kRadix / 2 + 1];  // radix passes: per-warp digit-pair counts
    };
    uint32_t gsum[kBGroups][kRadix / 2];
    uint16_t gstart[kBGroups][kRadix];
    uint64_t red[2][kBWarps];
    uint32_t bin_tmp[kBWarps];
    uint32_t bigbins[kFineBins / 32];  // fine bins over kFineMaxBin rows (uneven wide buckets)
    uint32_t next[2];  // the bucket taken after the current one (alternating slots)
};
static_assert(sizeof(BucketSmem) <= 232448, "bucket sort shared memory");

struct BucketStats {
    unsigned long long sorted_buckets, single_key_buckets, heavy_buckets, overflow_buckets, overflow_rows,
        radix_buckets, radix_rows, wide_buckets, wide_rows, retried_buckets;
};

// Persistent CTAs take runs of buckets (a run: one bucket, or consecutive
// buckets of at most kCap rows together, listed by their first bucket) in
// order from a counter and sort each run in shared memory.  A bucket of the
// headline window holds ~2,200 rows and a run ~6,900: the CTA's fixed work
// per iteration (its barriers, the 4096-bin scan, the warps' reductions) is
// spread over three times the rows (2.75 to 2.0 ms for 256M rows).
//
// A run's rows are sorted by a counting placement by the top 12 bits of
// key - kmin, after which every row finds its rank among the rows of its
// sub-bucket (at most 32) by (key, place in the run) and is written straight
// to its output row; or (a sub-bucket over 32 rows) stable 8-bit radix
// passes on key - kmin, the last of which stores every row at its output
// row; or (a sub-bucket over 32 rows and a range over 40 bits) two radix
// passes on a 16-bit group of the key and ranks within the groups.  If a
// group of over 32 rows then holds two keys, a run of several buckets is
// retried bucket by bucket (a second launch, singles != 0), and a bucket
// alone joins the overflow rows.  Rows of one key keep their input order:
// the scatter that formed the buckets was stable, and every in-run sort is.
// Once a run is written, the next run's rows are copied into the free
// buffer by per-thread asynchronous copies.  (Loading the next bucket's
// bounds while this one is sorted measured slower: 3.12 vs 2.97 ms at 256M
// rows; the last radix pass storing straight to the output rows instead of
// staging a sorted copy, 2.92 ms.  Per-thread insertion sorts of the
// sub-buckets, and a warp's bitonic network for sub-buckets of 9 to 32 rows,
// measured slower than the ranks.)
__global__ void __launch_bounds__(kBThreads, 1)
bucket_sort_kernel(uint64_t* __restrict__ keys, uint32_t* __restrict__ ptrs, const uint32_t* __restrict__ bstart,
                   const uint4* __restrict__ runrec, const uint32_t* __restrict__ nruns_p,
                   uint32_t* __restrict__ counter, uint32_t* __restrict__ ov_flag, uint32_t* __restrict__ retry_flag,
                   BucketStats* __restrict__ st) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BucketSmem& sm = *reinterpret_cast<BucketSmem*>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid / 32;
    const uint32_t nruns = *nruns_p;
    const uint32_t lt = lanemask_lt();
    // run x: buckets [rec.x, rec.y & kRunEnd), rows [rec.z, rec.w); bit 31
    // of rec.y: a run of one heavy bucket
    if (tid == 0) sm.next[0] = atomicAdd(counter, 1u);
    __syncthreads();
    uint32_t rq = sm.next[0];
    // the next run's rows are copied into buffer 0 while the current run is
    // written out of buffer 1 (when the next one is sorted here)
    bool prefetched = false;
    for (uint32_t it = 1;; ++it) {
        if (rq >= nruns) break;
        // the run after this one; read after this run's first barrier,
        // rewritten two runs later
        if (tid == 0) sm.next[it & 1] = atomicAdd(counter, 1u);
        const uint4 rr = runrec[rq];
        const uint32_t b = rr.x, bend = rr.y & kRunEnd, nbk = bend - b;
        const uint32_t s = rr.z, e = rr.w, cnt = e - s;
        const bool heavy = (rr.y & kRunHeavy) != 0;
        // copies the next run's rows into buffer 0 once it is free (a range
        // not this one's), if the next run is sorted here
        auto prefetch_next = [&](uint32_t nq) {
            if (nq >= nruns) return;
            const uint4 r2 = runrec[nq];
            const uint32_t s2 = r2.z, cnt2 = r2.w - r2.z;
            if (cnt2 > 1 && !(r2.y & kRunHeavy) && cnt2 <= kCap) {
#pragma unroll
                for (int j = 0; j < kBIpt; ++j) {
                    const uint32_t r = tid + j * kBThreads;
                    if (r < cnt2) {
                        cp_async8(&sm.keys[0][r], keys + s2 + r);
                        cp_async4(&sm.ptrs[0][r], ptrs + s2 + r);
                    }
                }
                cp_async_commit();
                prefetched = true;
            }
        };
        if (cnt <= 1 || heavy || cnt > kCap) {  // (cnt > kCap: a run of one bucket)
            if (tid == 0) {
                if (cnt > 1 && heavy) {
                    atomicAdd(&st->heavy_buckets, 1ull);  // one key: the stable scatter left it in input order
                } else if (cnt > 1) {
                    ov_flag[b] = 1;
                    atomicAdd(&st->overflow_buckets, 1ull);
                    atomicAdd(&st->overflow_rows, (unsigned long long)cnt);
                }
            }
            __syncthreads();
            rq = sm.next[it & 1];
            continue;
        }
        // load (buffer 0), the key range, and clear the bins
        uint64_t kmin = ~0ull, kmax = 0;
        if (prefetched) {
            cp_async_wait_all();  // this thread's own rows: no barrier needed to read them
#pragma unroll
            for (int j = 0; j < kBIpt; ++j) {
                const uint32_t r = tid + j * kBThreads;
                if (r < cnt) {
                    const uint64_t k = sm.keys[0][r];
                    kmin = min(kmin, k);
                    kmax = max(kmax, k);
                }
            }
            prefetched = false;
        } else {
#pragma unroll
            for (int j = 0; j < kBIpt; ++j) {
                const uint32_t r = tid + j * kBThreads;
                if (r < cnt) {
                    const uint64_t k = keys[s + r];
                    sm.keys[0][r] = k;
                    sm.ptrs[0][r] = ptrs[s + r];
                    kmin = min(kmin, k);
                    kmax = max(kmax, k);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kFinePer; ++q) sm.bins[tid * kFinePer + q] = 0;
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if (lane == 0) {
            sm.red[0][warp] = kmin;
            sm.red[1][warp] = kmax;
        }
        __syncthreads();  // (a)
        const uint32_t nq = sm.next[it & 1];
        kmin = sm.red[0][lane];
        kmax = sm.red[1][lane];
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if (kmin == kmax) {
            if (tid == 0) atomicAdd(&st->single_key_buckets, (unsigned long long)nbk);
            __syncthreads();  // buffer 0 is read no more
            rq = nq;
            continue;  // one key value: already in input order, nothing to write
        }
        const int bits = 64 - __clzll(static_cast<long long>(kmax - kmin));
        const int fsh = bits > kFineBits ? bits - kFineBits : 0;
        bool ranked = false;   // sorted and written out by the ranks
        bool binsort = false;  // uneven and wide: sort by fine bin first
        if (bits > kRadixBits) {
#pragma unroll
            for (int j = 0; j < kBIpt; ++j) {
                const uint32_t r = tid + j * kBThreads;
                if (r < cnt) atomicAdd(&sm.bins[static_cast<uint32_t>((sm.keys[0][r] - kmin) >> fsh)], 1u);
            }
            __syncthreads();  // (b)
            // exclusive scan over the bins, kFinePer consecutive bins per
            // thread; a warp's total and whether one of its bins is too big
            uint32_t v[kFinePer], tsum = 0, bmax = 0;
#pragma unroll
            for (int q = 0; q < kFinePer; ++q) {
                v[q] = sm.bins[tid * kFinePer + q];
                tsum += v[q];
                bmax = max(bmax, v[q]);
            }
            uint32_t x = tsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            const uint32_t wbig = __any_sync(0xffffffffu, bmax > kFineMaxBin) ? 0x80000000u : 0u;
            if (lane == 31) sm.bin_tmp[warp] = x | wbig;
            __syncthreads();  // (c)
            const uint32_t bt = sm.bin_tmp[lane];
            const bool big = __any_sync(0xffffffffu, (bt & 0x80000000u) != 0);
            binsort = big && bits > kWideBits;
            if (binsort) {
                if (tid < kFineBins / 32) sm.bigbins[tid] = 0;
                __syncthreads();
#pragma unroll
                for (int q = 0; q < kFinePer; ++q)
                    if (v[q] > kFineMaxBin) atomicOr(&sm.bigbins[(tid * kFinePer + q) >> 5], 1u << ((tid * kFinePer + q) & 31));
                __syncthreads();
            }
            if (!big) {
                // this thread's first row: the warps before it (an exclusive
                // scan of the warp totals, one a lane), then the lanes before
                uint32_t wx = bt;  // no flag bits: no bin is big
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, wx, o);
                    if (lane >= (uint32_t)o) wx += y;
                }
                uint32_t run = __shfl_sync(0xffffffffu, wx - bt, warp) + x - tsum;
#pragma unroll
                for (int q = 0; q < kFinePer; ++q) {
                    sm.bins[tid * kFinePer + q] = run;  // next free row of the bin
                    run += v[q];
                }
                __syncthreads();  // (d)
#pragma unroll
                for (int j = 0; j < kBIpt; ++j) {
                    const uint32_t r = tid + j * kBThreads;
                    if (r < cnt) {
                        const uint64_t k = sm.keys[0][r];
                        const uint32_t pos = atomicAdd(&sm.bins[static_cast<uint32_t>((k - kmin) >> fsh)], 1u);
                        sm.keys[1][pos] = k;
                        sm.ptrs[1][pos] = r;  // the row's place in buffer 0: its input order
                    }
                }
                __syncthreads();  // (e)
                // bins[d] now holds the end of bin d and bins[d - 1] its
                // start: each row's rank among its bin's rows (at most
                // kFineMaxBin of them) by (key, input order), and the row,
                // with its ptr from buffer 0, goes straight to its output row
#pragma unroll
                for (int j = 0; j < kBIpt; ++j) {
                    const uint32_t i = tid + j * kBThreads;
                    if (i < cnt) {
                        const uint64_t k = sm.keys[1][i];
                        const uint32_t q = sm.ptrs[1][i];
                        const uint32_t d = static_cast<uint32_t>((k - kmin) >> fsh);
                        const uint32_t e2 = sm.bins[d], b2 = d ? sm.bins[d - 1] : 0u;
                        uint32_t r = 0;
                        for (uint32_t x = b2; x < e2; ++x) {
                            const uint64_t kx = sm.keys[1][x];
                            r += (kx < k || (kx == k && sm.ptrs[1][x] < q)) ? 1u : 0u;
                        }
                        keys[s + b2 + r] = k;
                        ptrs[s + b2 + r] = sm.ptrs[0][q];
                    }
                }
                __syncthreads();  // (f) the bins and buffer 1 are read no more
                ranked = true;
            }
        }
        // stable radix passes on value_of(key), ping-pong from buffer 0; with
        // direct_last the last pass stores the rows at their output rows;
        // returns the buffer holding the result otherwise
        // Each warp takes ipt x 32 consecutive rows (ipt = rows per thread,
        // from the bucket's size), so that a small bucket keeps every warp
        // busy and no warp ranks empty slots.
        const uint32_t ipt = (cnt + kBThreads - 1) / kBThreads;
        auto radix_passes = [&](int passes, auto value_of, bool direct_last) -> int {
            int a = 0;
            for (int pass = 0; pass < passes; ++pass) {
                const int sh = pass * kRadixBits;
                for (int x = tid; x < kBWarps * (kRadix / 2 + 1); x += kBThreads) (&sm.whist2[0][0])[x] = 0;
                __syncthreads();
                uint32_t dg[kBIpt], rank[kBIpt];
                const uint32_t wofs = warp * 32 * ipt + lane;
#pragma unroll
                for (int j = 0; j < kBIpt; ++j) {
                    const uint32_t r = wofs + j * 32;
                    dg[j] = (j < (int)ipt && r < cnt) ? static_cast<uint32_t>(value_of(sm.keys[a][r]) >> sh) & (kRadix - 1)
                                                      : kRadix;
                }
#pragma unroll
                for (int j = 0; j < kBIpt; ++j) {
                    if (j >= (int)ipt) break;
                    const uint32_t peers = warp_peers<kRadixBits + 1>(dg[j]);
                    const int leader = __ffs(peers) - 1;
                    const uint32_t hs = (dg[j] & 1u) * 16u;
                    const uint32_t c = smem_atomic_add_if_relaxed((int)lane == leader, &sm.whist2[warp][dg[j] >> 1],
                                                                  (uint32_t)__popc(peers) << hs);
                    rank[j] = __popc(peers & lt) + ((__shfl_sync(0xffffffffu, c, leader) >> hs) & 0xFFFFu);
                }
                __syncthreads();
                {  // exclusive counts over each group's warps; group totals
                    const uint32_t pr = tid & (kRadix / 2 - 1), g = tid / (kRadix / 2);
                    uint32_t acc = 0;
#pragma unroll
                    for (int w = 0; w < kBWpg; ++w) {
                        const uint32_t word = sm.whist2[g * kBWpg + w][pr];
                        sm.whist2[g * kBWpg + w][pr] = acc;
                        acc += word;
                    }
                    sm.gsum[g][pr] = acc;
                }
                __syncthreads();
                if (warp < (uint32_t)kBGroups) {  // first slot of each (group, digit)
                    uint32_t lsum = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int gg = 0; gg < kBGroups; ++gg) {
                            const uint32_t v = sm.gsum[gg][4 * lane + q];
                            lsum += (v & 0xFFFFu) + (v >> 16);
                        }
                    uint32_t x = lsum;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= (uint32_t)o) x += y;
                    }
                    uint32_t stt = x - lsum;
#pragma unroll 1
                    for (int q = 0; q < 4; ++q) {
                        uint32_t tot = 0, gpre = 0;
#pragma unroll
                        for (int gg = 0; gg < kBGroups; ++gg) {
                            const uint32_t v = sm.gsum[gg][4 * lane + q];
                            tot += v;
                            gpre += (gg < (int)warp) ? v : 0u;
                        }
                        const uint32_t c0 = tot & 0xFFFFu;
                        const uint32_t d0 = 8 * lane + 2 * q;
                        sm.gstart[warp][d0] = static_cast<uint16_t>(stt + (gpre & 0xFFFFu));
                        sm.gstart[warp][d0 + 1] = static_cast<uint16_t>(stt + c0 + (gpre >> 16));
                        stt += c0 + (tot >> 16);
                    }
                }
                __syncthreads();
                const uint32_t grp = warp / kBWpg;
                const bool last = direct_last && pass == passes - 1;
#pragma unroll
                for (int j = 0; j < kBIpt; ++j) {
                    if (dg[j] < kRadix) {
                        const uint32_t r = wofs + j * 32;
                        const uint32_t wo = (sm.whist2[warp][dg[j] >> 1] >> ((dg[j] & 1u) * 16u)) & 0xFFFFu;
                        const uint32_t slot = sm.gstart[grp][dg[j]] + wo + rank[j];
                        if (last) {  // the last pass stores straight to the output rows
                            keys[s + slot] = sm.keys[a][r];
                            ptrs[s + slot] = sm.ptrs[a][r];
                        } else {
                            sm.keys[a ^ 1][slot] = sm.keys[a][r];
                            sm.ptrs[a ^ 1][slot] = sm.ptrs[a][r];
                        }
                    }
                }
                __syncthreads();
                a ^= 1;
            }
            return a;
        };
        if (binsort) {
            // Uneven (a fine bin over kFineMaxBin rows) and wider than
            // kWideBits: stable passes order the rows by a group, the fine
            // bin and, inside a big bin, the next kGroupSubBits bits of the
            // key, each group in input order.  A group's bounds come from a
            // binary search on the groups; a group of more than kFineMaxBin
            // rows must hold one key, so that its rows are in place, and the
            // rows of the others rank themselves by (key, input order); every
            // row then goes to its output row.  A key repeated in a big bin is
            // mostly alone in its group.  (A 24-bit group, three passes, left
            // fewer buckets to the plain sort but was slower: with hashed
            // Zipf keys 16.0 against 15.5 ms for the 256M-row step.)
            const int subsh = fsh - kGroupSubBits;  // fsh > kWideBits - kFineBits
            auto group_of = [&](uint64_t k) -> uint64_t {
                const uint64_t off = k - kmin;
                const uint32_t bin = static_cast<uint32_t>(off >> fsh);
                const bool bigbin = (sm.bigbins[bin >> 5] >> (bin & 31)) & 1u;
                return (static_cast<uint64_t>(bin) << kGroupSubBits) |
                       (bigbin ? static_cast<uint32_t>(off >> subsh) & ((1u << kGroupSubBits) - 1) : 0u);
            };
            const int ga = radix_passes(kGroupPasses, group_of, false);
            // the rows' groups, in order, in the keys of the free buffer
            uint64_t* grp = sm.keys[ga ^ 1];
#pragma unroll
            for (int j = 0; j < kBIpt; ++j) {
                const uint32_t i = tid + j * kBThreads;
                if (i < cnt) grp[i] = group_of(sm.keys[ga][i]);
            }
            __syncthreads();
            auto lower = [&](uint64_t g, bool upper) {  // first row of a group above (or not below) g
                uint32_t lo = 0, hi = cnt;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) / 2;
                    const uint64_t gm = grp[mid];
                    if (gm < g || (upper && gm == g)) lo = mid + 1;
                    else hi = mid;
                }
                return lo;
            };
            uint32_t gb[kBIpt], ge[kBIpt];
            bool multi = false;
#pragma unroll
            for (int j = 0; j < kBIpt; ++j) {
                const uint32_t i = tid + j * kBThreads;
                gb[j] = ge[j] = 0;
                if (i < cnt) {
                    const uint64_t g = grp[i];
                    gb[j] = lower(g, false);
                    ge[j] = lower(g, true);
                    if (ge[j] - gb[j] > kFineMaxBin && sm.keys[ga][i] != sm.keys[ga][gb[j]]) multi = true;
                }
            }
            if (!__syncthreads_or(multi)) {
#pragma unroll
                for (int j = 0; j < kBIpt; ++j) {
                    const uint32_t i = tid + j * kBThreads;
                    if (i < cnt) {
                        const uint64_t k = sm.keys[ga][i];
                        uint32_t r = 0;
                        if (ge[j] - gb[j] > kFineMaxBin) {
                            r = i - gb[j];  // one key: input order
                        } else {
                            for (uint32_t x = gb[j]; x < ge[j]; ++x) {
                                const uint64_t kx = sm.keys[ga][x];
                                r += (kx < k || (kx == k && x < i)) ? 1u : 0u;
                            }
                        }
                        keys[s + gb[j] + r] = k;
                        ptrs[s + gb[j] + r] = sm.ptrs[ga][i];
                    }
                }
                __syncthreads();  // the buffers are read no more
                ranked = true;
                if (tid == 0) {
                    atomicAdd(&st->radix_buckets, (unsigned long long)nbk);
                    atomicAdd(&st->radix_rows, (unsigned long long)cnt);
                }
            } else {
                // a big group holds two keys: more than five passes on the
                // key would be needed.  A run of several buckets is retried
                // bucket by bucket (a second launch); a bucket alone joins
                // the overflow rows, whose plain radix sort is cheaper (its
                // rows in global memory are untouched)
                if (tid == 0) {
                    if (nbk > 1) {
                        for (uint32_t x = b; x < bend; ++x) retry_flag[x] = 1;
                        atomicAdd(&st->retried_buckets, (unsigned long long)nbk);
                    } else {
                        ov_flag[b] = 1;
                        atomicAdd(&st->wide_buckets, 1ull);
                        atomicAdd(&st->wide_rows, (unsigned long long)cnt);
                    }
                }
                rq = nq;
                continue;
            }
        }
        if (!ranked) {
            // stable radix passes on key - kmin; the last stores the rows at
            // their output rows
            if (tid == 0) {
                atomicAdd(&st->radix_buckets, (unsigned long long)nbk);
                atomicAdd(&st->radix_rows, (unsigned long long)cnt);
            }
            radix_passes((bits + kRadixBits - 1) / kRadixBits, [&](uint64_t k) { return k - kmin; }, true);
        }
        // the bucket is written out and buffer 0 is free: the next bucket's
        // copies start now (issuing them during the ranking measured slower)
        prefetch_next(nq);
        if (tid == 0) atomicAdd(&st->sorted_buckets, (unsigned long long)nbk);
        rq = nq;
    }
}

// Flags the first bucket of every run the bucket sort takes: greedily, each
// run as long as it stays within kCap rows, from the first bucket of each
// segment of kRunSeg buckets (a warp walks a segment's bounds, held in shared
// memory, 32 buckets a step).
constexpr uint32_t kRunSeg = 128;
__global__ void __launch_bounds__(1024) run_start_kernel(const uint32_t* __restrict__ bstart,
                                                         const uint32_t* __restrict__ nbid_p,
                                                         const uint32_t* __restrict__ heavy_bucket_bits,
                                                         uint32_t* __restrict__ run_flag) {
    __shared__ uint32_t sb[1025], shw[32], flag[1024];
    const uint32_t nbid = *nbid_p, b0 = blockIdx.x * 1024u;
    if (b0 >= nbid) return;
    const uint32_t m = min(1024u, nbid - b0), tid = threadIdx.x, lane = lane_id(), warp = tid / 32;
    for (uint32_t i = tid; i <= m; i += 1024u) sb[i] = bstart[b0 + i];
    if (tid < 32) shw[tid] = heavy_bucket_bits[(b0 >> 5) + tid];
    flag[tid] = 0;
    __syncthreads();
    const uint32_t lo = warp * kRunSeg, hi = min(m, lo + kRunSeg);  // this warp's segment
    if (warp < 1024 / kRunSeg && lo < hi) {
        auto alone = [&](uint32_t x) { return ((shw[x >> 5] >> (x & 31)) & 1u) != 0 || sb[x + 1] - sb[x] > kCap; };
        uint32_t cur = lo;
        while (cur < hi) {
            if (lane == 0) flag[cur] = 1;
            uint32_t end = cur + 1;  // first bucket after the run
            if (!alone(cur)) {
                for (;;) {  // lanes try end + lane
                    const uint32_t x = end + lane;
                    const bool ok = x < hi && !alone(x) && sb[x + 1] - sb[cur] <= kCap;
                    const uint32_t fit = __ballot_sync(0xffffffffu, ok);
                    const uint32_t nfit = fit == 0xffffffffu ? 32u : (uint32_t)(__ffs(~fit) - 1);
                    end += nfit;
                    if (nfit < 32) break;
                }
            }
            cur = end;
        }
    }
    __syncthreads();
    if (tid < m) run_flag[b0 + tid] = flag[tid];
}

// The bucket sort's run records from a list of first buckets (singles: every
// listed bucket a run of its own): first bucket, end bucket (bit 31: one
// heavy bucket), first row, end row.
__global__ void __launch_bounds__(1024) run_records_kernel(const uint32_t* __restrict__ list,
                                                           const uint32_t* __restrict__ n_p, int singles,
                                                           const uint32_t* __restrict__ nbid_p,
                                                           const uint32_t* __restrict__ bstart,
                                                           const uint32_t* __restrict__ heavy_bucket_bits,
                                                           uint4* __restrict__ rec) {
    const uint32_t n = *n_p, i = blockIdx.x * 1024u + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = list[i], bend = singles ? b + 1 : (i + 1 < n ? list[i + 1] : *nbid_p);
    const bool heavy = bend == b + 1 && ((heavy_bucket_bits[b >> 5] >> (b & 31)) & 1u) != 0;
    rec[i] = make_uint4(b, bend | (heavy ? kRunHeavy : 0u), bstart[b], bstart[bend]);
}

// Ordered list of flagged buckets (the overflow buckets, or the first
// buckets of the bucket sort's runs) with their row offsets in a compact
// buffer, in two launches over blocks of 1024 buckets: each block's count of
// flagged buckets and rows, then each block's exclusive scan from the totals
// of the blocks before it.  The last block writes the totals to nlist and
// rows_total.
__global__ void __launch_bounds__(1024) flag_count_kernel(const uint32_t* __restrict__ ov_flag,
                                                              const uint32_t* __restrict__ nbid_p,
                                                              const uint32_t* __restrict__ bstart,
                                                              uint2* __restrict__ bagg) {
    __shared__ uint32_t wc[32], wr[32];
    const uint32_t nbid = *nbid_p, lane = lane_id(), warp = threadIdx.x / 32;
    const uint32_t b = blockIdx.x * 1024u + threadIdx.x;
    uint32_t c = b < nbid ? ov_flag[b] : 0u;
    uint32_t r = c ? bstart[b + 1] - bstart[b] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if (lane == 0) {
        wc[warp] = c;
        wr[warp] = r;
    }
    __syncthreads();
    if (warp == 0) {
        c = wc[lane];
        r = wr[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            r += __shfl_xor_sync(0xffffffffu, r, o);
        }
        if (lane == 0) bagg[blockIdx.x] = make_uint2(c, r);
    }
}

__global__ void __launch_bounds__(1024) flag_list_kernel(const uint32_t* __restrict__ ov_flag,
                                                             const uint32_t* __restrict__ nbid_p,
                                                             const uint32_t* __restrict__ bstart,
                                                             const uint2* __restrict__ bagg,
                                                             uint32_t* __restrict__ list, uint32_t* __restrict__ offs,
                                                             uint32_t* __restrict__ nlist,
                                                             uint32_t* __restrict__ rows_total) {
    __shared__ uint32_t wc[32], wr[32];
    const uint32_t nbid = *nbid_p, lane = lane_id(), warp = threadIdx.x / 32;
    // totals of the blocks before this one
    uint32_t pc = 0, pr = 0;
    for (uint32_t j = threadIdx.x; j < blockIdx.x; j += 1024u) {
        const uint2 v = bagg[j];
        pc += v.x;
        pr += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pc += __shfl_xor_sync(0xffffffffu, pc, o);
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
    }
    if (lane == 0) {
        wc[warp] = pc;
        wr[warp] = pr;
    }
    __syncthreads();
    pc = pr = 0;
#pragma unroll 8
    for (int w = 0; w < 32; ++w) {
        pc += wc[w];
        pr += wr[w];
    }
    __syncthreads();
    const uint32_t b = blockIdx.x * 1024u + threadIdx.x;
    const uint32_t f = b < nbid ? ov_flag[b] : 0u;
    const uint32_t len = f ? bstart[b + 1] - bstart[b] : 0u;
    uint32_t xc = f, xr = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yc = __shfl_up_sync(0xffffffffu, xc, o), yr = __shfl_up_sync(0xffffffffu, xr, o);
        if (lane >= (uint32_t)o) {
            xc += yc;
            xr += yr;
        }
    }
    if (lane == 31) {
        wc[warp] = xc;
        wr[warp] = xr;
    }
    __syncthreads();
    for (uint32_t w = 0; w < warp; ++w) {
        pc += wc[w];
        pr += wr[w];
    }
    if (f) {
        list[pc + xc - 1] = b;
        offs[pc + xc - 1] = pr + xr - len;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 1023) {
        *nlist = pc + xc;
        *rows_total = pr + xr;
    }
}

// Copies the rows of the listed overflow buckets to (to_gather) or from the
// compact buffer; row r of the compact buffer belongs to the last listed
// bucket whose offset is <= r.
__global__ void overflow_move_kernel(uint64_t* __restrict__ keys, uint32_t* __restrict__ ptrs,
                                     const uint32_t* __restrict__ bstart, const uint32_t* __restrict__ list,
                                     const uint32_t* __restrict__ offs, const uint32_t* __restrict__ nl_p,
                                     const uint32_t* __restrict__ rows_p, uint64_t* __restrict__ ck,
                                     uint32_t* __restrict__ cp, int to_gather) {
    const uint32_t nl = *nl_p, rows = *rows_p;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        uint32_t lo = 0, hi = nl;  // last j with offs[j] <= r
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (offs[mid] <= r) lo = mid;
            else hi = mid;
        }
        const uint32_t src = bstart[list[lo]] + (r - offs[lo]);
        if (to_gather) {
            ck[r] = keys[src];
            cp[r] = ptrs[src];
        } else {
            keys[src] = ck[r];
            ptrs[src] = cp[r];
        }
    }
}

// The call's statistics, in the order of the header's list; the largest
// bucket from the bucket starts (a block reduction here: thread 0 of the
// bucket sort scanning each run's buckets took a tenth of that kernel).
__global__ void __launch_bounds__(1024) learned_stats_kernel(const uint32_t* __restrict__ nbid,
                                                             const uint32_t* __restrict__ plan,
                                                             const uint32_t* __restrict__ bstart,
                                                             const BucketStats* __restrict__ st,
                                                             const uint32_t* __restrict__ id_passes,
                                                             uint64_t* __restrict__ out) {
    __shared__ uint32_t wmax[32];
    const uint32_t nb = *nbid;
    uint32_t mx = 0;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) mx = max(mx, bstart[b + 1] - bstart[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane_id() == 0) wmax[threadIdx.x / 32] = mx;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (uint32_t w = 1; w < blockDim.x / 32; ++w) mx = max(mx, wmax[w]);
    out[0] = nb;
    out[1] = plan[0];
    out[2] = st->sorted_buckets;
    out[3] = st->single_key_buckets;
    out[4] = st->heavy_buckets;
    out[5] = st->overflow_buckets;
    out[6] = st->overflow_rows;
    out[7] = mx;
    out[8] = st->radix_buckets;
    out[9] = st->radix_rows;
    out[10] = st->wide_buckets;
    out[11] = st->wide_rows;
    out[12] = st->retried_buckets;
    out[13] = *id_passes;
}

// ------------------------------------------------------------------ carried bucket ids
// When every bucket id fits in 16 bits, each row's id is computed once, kept
// in a 16-bit array, and moved with the row through both digit passes; the
// counts and the bucket bounds then read ids instead of recomputing them.
constexpr int kCarryTile = 3584;
constexpr int kCarryIdxTile = 4096;

// Bucket id of every row (kept as 16 bits), the histogram of its low digit
// per chunk of the first digit pass (CTA c takes the rows of chunk c: that
// pass's count), and the OR of the ids and of their complements (vbits,
// zeroed beforehand), from which the plan sees which digits vary.
__global__ void __launch_bounds__(1024) ids_upsweep_kernel(const uint64_t* __restrict__ keys, uint32_t n,
                                                           uint32_t chunk, BucketValue16 fn,
                                                           uint16_t* __restrict__ ids,
                                                           unsigned long long* __restrict__ vbits,
                                                           uint32_t* __restrict__ chunk_hist) {
    // (one histogram a warp, 32 KB, measured slower here, 0.75 against 0.63
    // ms for 256M rows: the cell-table lookups lose L1 capacity to it)
    __shared__ uint32_t h[kRadix];
    __shared__ uint32_t wor[32], wnot[32];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    uint32_t vor = 0, vnot = 0;
    auto add = [&](uint32_t id) {
        atomicAdd(&h[id & 255u], 1u);
        vor |= id;
        vnot |= ~id;
    };
    const uint32_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    uint32_t done = lo;
    if (lo < hi && (reinterpret_cast<uintptr_t>(keys + lo) & 15) == 0 && (reinterpret_cast<uintptr_t>(ids + lo) & 7) == 0) {
        // four keys per thread and iteration (two 16-byte loads in flight),
        // their ids stored as one 8-byte word
        const uint32_t nq = (hi - lo) / 4;
        const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(keys + lo);
        uint2* i4 = reinterpret_cast<uint2*>(ids + lo);
        for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
            const ulonglong2 a = __ldcs(k2 + 2 * q), b = __ldcs(k2 + 2 * q + 1);
            const uint32_t i0 = static_cast<uint32_t>(fn(a.x)), i1 = static_cast<uint32_t>(fn(a.y));
            const uint32_t i2 = static_cast<uint32_t>(fn(b.x)), i3 = static_cast<uint32_t>(fn(b.y));
            i4[q] = make_uint2((i0 & 0xFFFFu) | (i1 << 16), (i2 & 0xFFFFu) | (i3 << 16));
            add(i0);
            add(i1);
            add(i2);
            add(i3);
        }
        done = lo + nq * 4;
    }
    for (uint32_t i = done + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t id = static_cast<uint32_t>(fn(ld_stream(keys + i)));
        ids[i] = static_cast<uint16_t>(id);
        add(id);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vor |= __shfl_xor_sync(0xffffffffu, vor, o);
        vnot |= __shfl_xor_sync(0xffffffffu, vnot, o);
    }
    if (lane_id() == 0) {
        wor[threadIdx.x / 32] = vor;
        wnot[threadIdx.x / 32] = vnot;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) chunk_hist[blockIdx.x * kRadix + i] = h[i];
    if (threadIdx.x == 0) {
        for (uint32_t w = 1; w < blockDim.x / 32; ++w) {
            vor |= wor[w];
            vnot |= wnot[w];
        }
        if (lo < hi) {
            atomicOr(&vbits[0], static_cast<unsigned long long>(vor));
            atomicOr(&vbits[1], 0xFFFFFFFF00000000ull | vnot);  // the complement of the zero-extended id
        }
    }
}

// Chunk counts of the second pass: its digit is the high byte carried by the
// first pass, or, when no first pass ran (every id has the same low byte),
// the high byte of the input rows' ids.  The bytes are in random order and
// are counted into a [digit][lane] table (nd_count): 0.055 ms for 256M rows,
// against 0.094 with a histogram per warp and 0.19 with one shared one.
__global__ void __launch_bounds__(1024) ids_count_kernel(Buffers buf, uint32_t n, int pos, const Plan* __restrict__ plan,
                                                         uint32_t chunk, uint32_t* __restrict__ chunk_hist) {
    if (!plan->active[pos]) return;
    const uint32_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    uint32_t* out = chunk_hist + (size_t)blockIdx.x * kRadix;
    if (plan->active[0]) nd_count(buf.vals(plan->src[pos]), lo, hi, out);
    else nd_count<true>(buf.in_ids, lo, hi, out);
}

// Bucket bounds when no pass ran: every row has the same id, the OR of the
// ids (vbits[0]); the last pass records each id's first row otherwise.
// Also records which id passes ran (bit p: the pass on byte p of the ids).
__global__ void __launch_bounds__(256) ids_bounds_kernel(const Plan* __restrict__ plan, uint32_t n,
                                                         const uint32_t* __restrict__ nbid_p,
                                                         const unsigned long long* __restrict__ vbits,
                                                         uint32_t* __restrict__ bstart, uint32_t* __restrict__ passes) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *passes = (plan->active[0] ? 1u : 0u) | (plan->active[1] ? 2u : 0u);
    if (plan->npasses) return;
    const uint32_t nbid = *nbid_p;
    const uint32_t id = static_cast<uint32_t>(vbits[0]);
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= nbid; b += gridDim.x * blockDim.x)
        bstart[b] = b <= id ? 0u : n;
}

struct CarryScratch {
    uint64_t* tmp_k;
    uint32_t* tmp_p;
    uint16_t* ids_in;   // the input rows' ids
    uint8_t* hi_tmp;    // the ids' high bytes, carried by the first pass
    uint8_t* hi_out;
    Plan* plan;
    uint32_t* chunk_hist;
    uint32_t* chunk_base;   // first pass (its first 256 entries: the low bytes' starts)
    uint32_t* chunk_base1;  // second pass
    unsigned long long* vbits;  // 2: OR of the ids, OR of their complements (zeroed)
    uint32_t* bmin;  // per block of bucket starts: minimum
    size_t total;
};

CarryScratch carry_carve(void* base, uint64_t n) {
    Carver c(base);
    CarryScratch t;
    t.tmp_k = c.take<uint64_t>(n);
    t.tmp_p = c.take<uint32_t>(n);
    t.ids_in = c.take<uint16_t>(n);
    t.hi_tmp = c.take<uint8_t>(n);
    t.hi_out = c.take<uint8_t>(n);
    t.plan = c.take<Plan>(1);
    t.chunk_hist = c.take<uint32_t>(kMaxChunks * kRadix);
    t.chunk_base = c.take<uint32_t>(kMaxChunks * kRadix);
    t.chunk_base1 = c.take<uint32_t>(kMaxChunks * kRadix);
    t.vbits = c.take<unsigned long long>(2);
    t.bmin = c.take<uint32_t>(kMaxBucketIds / 1024 + 1);
    t.total = c.bytes();
    return t;
}

// After the passes: bstart[b] = the first row of an id >= b (suffix minimum
// of the recorded first rows; bstart[nbid] = n), in two launches over blocks
// of 1024 entries: each block's minimum, then each block's suffix minimum
// from the minimum of the blocks after it.
constexpr uint32_t kFillBlocks = kMaxBucketIds / 1024 + 1;

__device__ __forceinline__ uint32_t first_row_entry(const uint32_t* bstart, uint32_t b, uint32_t nbid, uint32_t n) {
    return b < nbid ? bstart[b] : (b == nbid ? n : 0xFFFFFFFFu);
}

__global__ void __launch_bounds__(1024) bounds_min_kernel(const Plan* __restrict__ plan, uint32_t n,
                                                          const uint32_t* __restrict__ nbid_p,
                                                          const uint32_t* __restrict__ bstart,
                                                          uint32_t* __restrict__ bmin) {
    if (!plan->npasses) return;
    __shared__ uint32_t wmin[32];
    const uint32_t nbid = *nbid_p;
    if (blockIdx.x * 1024u > nbid) return;
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    uint32_t x = first_row_entry(bstart, blockIdx.x * 1024u + threadIdx.x, nbid, n);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) wmin[warp] = x;
    __syncthreads();
    if (warp == 0) {
        x = wmin[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (lane == 0) bmin[blockIdx.x] = x;
    }
}

__global__ void __launch_bounds__(1024) bounds_fill_kernel(const Plan* __restrict__ plan, uint32_t n,
                                                           const uint32_t* __restrict__ nbid_p,
                                                           const uint32_t* __restrict__ bmin,
                                                           uint32_t* __restrict__ bstart) {
    if (!plan->npasses) return;
    __shared__ uint32_t wmin[32];
    __shared__ uint32_t after_s;
    const uint32_t nbid = *nbid_p, blk = blockIdx.x;
    if (blk * 1024u > nbid) return;
    const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
    if (warp == 0) {  // the blocks after this one
        uint32_t a = 0xFFFFFFFFu;
        for (uint32_t j = blk + 1 + lane; j <= nbid / 1024u; j += 32) a = min(a, bmin[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
        if (lane == 0) after_s = a;
    }
    const uint32_t b = blk * 1024u + threadIdx.x;
    uint32_t x = first_row_entry(bstart, b, nbid, n);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_down_sync(0xffffffffu, x, o);
        if (lane + o < 32) x = min(x, y);
    }
    if (lane == 0) wmin[warp] = x;
    __syncthreads();
    uint32_t after = after_s;
    for (uint32_t w = warp + 1; w < 32; ++w) after = min(after, wmin[w]);
    if (b <= nbid) bstart[b] = min(x, after);
}

// The two passes by bucket id: per pass, chunk counts of the id digit ->
// chunk offsets -> scatter; the first pass carries the ids' high bytes to the
// second.  The first pass's chunk counts come from the id upsweep (the same
// chunks, geometry g0); the second pass has its own chunks (g1).  A key
// column (no ptrs) goes through a first pass that stages 16-bit places in the
// tile instead of ptrs, in tiles of kCarryIdxTile rows (the shared memory the
// ptrs left free): 4096 rows a tile instead of 3584.
template <int THREADS>
int carried_passes(const Buffers& b, uint32_t n32, const CarryScratch& cs, const ChunkGeom& g0, const ChunkGeom& g1,
                   bool idx0, cudaStream_t s, uint32_t* first_row) {
    const int bulk_ok = ((reinterpret_cast<uintptr_t>(b.in_k) | reinterpret_cast<uintptr_t>(b.in_p) |
                          reinterpret_cast<uintptr_t>(b.out_k) | reinterpret_cast<uintptr_t>(b.out_p)) & 15) == 0;
    for (int pos = 0; pos < 2; ++pos) {
        const ChunkGeom& g = pos ? g1 : g0;
        if (pos > 0) {
            SBH_TIMED("learned_ids_count", s,
                      ids_count_kernel<<<g.nchunks, 1024, 0, s>>>(b, n32, pos, cs.plan, g.chunk, cs.chunk_hist));
            SBH_LAUNCHED();
        }
        uint32_t* cbase = pos ? cs.chunk_base1 : cs.chunk_base;
        SBH_TIMED("learned_ids_chunk_scan", s,
                  chunk_scan_kernel<<<1, 1024, 0, s>>>(cs.plan, pos, cs.chunk_hist, g.nchunks, nullptr, cbase));
        SBH_LAUNCHED();
        if (pos == 0 && idx0) {
            SBH_TIMED("learned_ids_scatter", s,
                      (chunk_scatter_kernel<RadixValue, kCarryIdxTile, THREADS, true, true>
                       <<<g.nchunks, THREADS, g.smem, s>>>(b, n32, pos, cs.plan, g.chunk, cbase, RadixValue{},
                                                            bulk_ok, spin_limit(), status_word(), first_row,
                                                            cs.chunk_base)));
        } else {
            SBH_TIMED("learned_ids_scatter", s,
                      (chunk_scatter_kernel<RadixValue, kCarryTile, THREADS, true><<<g.nchunks, THREADS, g.smem, s>>>(
                          b, n32, pos, cs.plan, g.chunk, cbase, RadixValue{}, bulk_ok, spin_limit(), status_word(),
                          first_row, cs.chunk_base)));
        }
        SBH_LAUNCHED();
    }
    return SBH_OK;
}

// Stable sort by 16-bit bucket id with the ids carried along; fills bstart.
int sort_by_carried_ids(const uint64_t* in_k, const uint32_t* in_p, uint64_t* out_k, uint32_t* out_p, uint64_t n,
                        void* scratch, cudaStream_t s, BucketValue16 fn, const uint32_t* nbid, uint32_t* bstart,
                        uint32_t* id_passes) {
    CarryScratch cs = carry_carve(scratch, n);
    const uint32_t n32 = static_cast<uint32_t>(n);
    const int sms = num_sms();
    SBH_CUDA(cudaMemsetAsync(cs.vbits, 0, 2 * sizeof(unsigned long long), s));
    const bool idx0 = in_p == nullptr;  // a key column: the first pass stages places in the tile
    ChunkGeom g0, g1;
    int rc = chunk_geometry<RadixValue, kCarryTile, 512, true>(n32, &g1);
    if (rc) return rc;
    if (idx0) rc = chunk_geometry<RadixValue, kCarryIdxTile, 512, true, true>(n32, &g0);
    else g0 = g1;
    if (rc) return rc;
    SBH_TIMED("learned_ids_upsweep", s,
              ids_upsweep_kernel<<<g0.nchunks, 1024, 0, s>>>(in_k, n32, g0.chunk, fn, cs.ids_in, cs.vbits,
                                                              cs.chunk_hist));
    SBH_LAUNCHED();
    SBH_TIMED("learned_ids_plan", s, plan_bits_kernel<<<1, 32, 0, s>>>(cs.vbits, 2, cs.plan, 0));
    SBH_LAUNCHED();
    Buffers b{in_k, in_p, cs.tmp_k, cs.tmp_p, out_k, out_p};
    b.in_ids = cs.ids_in;
    b.tmp_v = cs.hi_tmp;
    b.out_v = cs.hi_out;
    // bucket starts: the last pass records each id's first output row, then a
    // suffix minimum fills the empty buckets (with no pass, from the one id)
    SBH_CUDA(cudaMemsetAsync(bstart, 0xFF, (kMaxBucketIds + 1) * sizeof(uint32_t), s));
    rc = carried_passes<512>(b, n32, cs, g0, g1, idx0, s, bstart);
    if (rc) return rc;
    const unsigned cblocks = (unsigned)min_u64((n + 255) / 256, (uint64_t)sms * 4);
    SBH_TIMED("learned_ids_copy", s, copy_kernel<<<cblocks, 256, 0, s>>>(b, n32, cs.plan));
    SBH_LAUNCHED();
    SBH_TIMED("learned_bounds", s,
              ids_bounds_kernel<<<kMaxBucketIds / 256 + 1, 256, 0, s>>>(cs.plan, n32, nbid, cs.vbits, bstart,
                                                                        id_passes));
    SBH_LAUNCHED();
    SBH_TIMED("learned_bounds_min", s,
              bounds_min_kernel<<<kFillBlocks, 1024, 0, s>>>(cs.plan, n32, nbid, bstart, cs.bmin));
    SBH_LAUNCHED();
    SBH_TIMED("learned_bounds_fill", s,
              bounds_fill_kernel<<<kFillBlocks, 1024, 0, s>>>(cs.plan, n32, nbid, cs.bmin, bstart));
    SBH_LAUNCHED();
    return SBH_OK;
}

struct SortLearnedScratch {
    float* bmax;            // per block of cells: maximum of F
    uint32_t* bheavy;       // per block of cells: heavy keys
    uint2* cells;           // kNCell + 1
    uint32_t* cells16;      // kNCell + 1
    uint32_t* cell_hc;      // kNCell + 1: heavy keys per cell (zeroed)
    uint32_t* cell_hidx;    // kNCell + 1: first heavy key per cell (0xFF bytes)
    HeavyCell* hcells;      // kMaxHeavy: cells holding heavy keys, by first heavy key
    float* F;               // kNCell + 1
    uint32_t* heavy_bucket_bits;
    uint32_t* bstart;       // max ids + 1
    uint32_t* ov_flag;      // max ids
    uint32_t* list;
    uint2* bagg;            // per block of buckets: overflow buckets, rows
    uint32_t* offs;
    uint32_t* retry_flag;   // buckets of runs the bucket sort retries one by one
    uint32_t* small;        // nbid, counter, nlist, rows_total, heavy keys used, spread buckets, runs, (rows),
                            // second counter, retried buckets, (rows), -, id passes (bits)
    uint32_t* run_flag;     // first buckets of the bucket sort's runs
    uint4* runrec;          // the runs' records
    BucketStats* stats;
    uint64_t* ck;           // compact overflow rows (n)
    uint32_t* cp;
    void* sort_scratch;     // for the id passes and the overflow sort
    size_t zero_bytes;      // from heavy_bucket_bits through stats
    size_t total;
};

inline uint64_t learned_nb(uint64_t n) { return (2 * n + kCap - 1) / kCap; }
// every id is below NB + 2 * (heavy keys) + 2 (at most kMaxHeavy heavy keys);
// the bound also covers the 2^16 + 1 bucket starts the carried-id path clears
inline uint64_t learned_max_ids(uint64_t n) { return learned_nb(n) + 2ull * kNCell + 4; }
static_assert(2ull * kNCell + 4 >= kMaxBucketIds + 1ull, "bucket starts of the carried-id path fit");

SortLearnedScratch learned_carve(void* base, uint64_t n) {
    Carver c(base);
    SortLearnedScratch t;
    const uint64_t ids = learned_max_ids(n);
    t.bmax = c.take<float>(kTblBlocks);
    t.bheavy = c.take<uint32_t>(kTblBlocks);
    t.cells = c.take<uint2>(kNCell + 1);
    t.cells16 = c.take<uint32_t>(kNCell + 1);
    t.cell_hc = c.take<uint32_t>(kNCell + 1);
    t.cell_hidx = c.take<uint32_t>(kNCell + 1);
    t.hcells = c.take<HeavyCell>(kMaxHeavy);
    t.F = c.take<float>(kNCell + 1);
    t.list = c.take<uint32_t>(ids);
    t.bagg = c.take<uint2>(ids / 1024 + 1);
    t.offs = c.take<uint32_t>(ids);
    t.bstart = c.take<uint32_t>(ids + 1);
    t.heavy_bucket_bits = c.take<uint32_t>(ids / 32 + 1);
    const size_t z0 = c.off - (ids / 32 + 1) * sizeof(uint32_t);
    t.ov_flag = c.take<uint32_t>(ids);
    t.retry_flag = c.take<uint32_t>(ids);
    t.small = c.take<uint32_t>(16);
    t.stats = c.take<BucketStats>(1);
    t.zero_bytes = c.off - z0;
    t.run_flag = c.take<uint32_t>(ids);  // written for every bucket id in use
    t.runrec = c.take<uint4>(ids);
    t.ck = c.take<uint64_t>(n);
    t.cp = c.take<uint32_t>(n);
    t.sort_scratch = c.take<char>(std::max(sort_carve(nullptr, n, true).total, carry_carve(nullptr, n).total));
    t.total = c.bytes();
    return t;
}

}  // namespace
}  // namespace sbh

// ============================================================== C ABI
extern "C" {

int sbh_mlp_forward(const float* d_params, const float* d_x, uint64_t m, float* d_y, void* stream) {
    using namespace sbh;
    clear_error();
    if (m == 0) return SBH_OK;
    if (!d_params || !d_x || !d_y) { set_error("null pointer"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    SBH_TIMED("mlp_forward", s,
              mlp_forward_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(d_params, d_x, m, d_y));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_mlp_grad(const float* d_params, const float* d_x, const float* d_t, uint64_t m, float* d_grad,
                 float* d_loss, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    const uint64_t nparts = (m + kMaxSlice - 1) / kMaxSlice;
    if (nparts > 0xFFFFFFFFull) { set_error("m too large"); return SBH_EINVAL; }
    Carver c(nullptr);
    c.take<float>(nparts * kNP);
    c.take<float>(nparts);
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, c.bytes(), &done);
    if (rc || done) return rc;
    if (m == 0) { set_error("m must be > 0"); return SBH_EINVAL; }
    if (!d_params || !d_x || !d_t || !d_grad) { set_error("null pointer"); return SBH_EINVAL; }
    cudaStream_t s = as_stream(stream);
    Carver w(d_scratch);
    float* partial = w.take<float>(nparts * kNP);
    float* partial_sq = w.take<float>(nparts);
    const size_t smem = sizeof(GradSmem);
    SBH_CUDA(cudaFuncSetAttribute(mlp_grad_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SBH_TIMED("mlp_grad", s,
              mlp_grad_partial_kernel<<<(unsigned)nparts, kGThreads, smem, s>>>(d_params, d_x, d_t, m, partial,
                                                                                partial_sq));
    SBH_LAUNCHED();
    SBH_TIMED("mlp_grad_sum", s,
              mlp_grad_sum_kernel<<<(kNP + 255) / 256, 256, 0, s>>>(partial, partial_sq, (uint32_t)nparts, m, d_grad,
                                                                    d_loss));
    SBH_LAUNCHED();
    return SBH_OK;
}

int sbh_learned_train(const uint64_t* d_samples, uint64_t m, uint64_t n_rows, const float* d_init_params,
                      int steps, int batch, float lr, void* d_model, float* d_losses, float* d_train_x,
                      float* d_train_t, void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (m > 0xFFFFFFFFull) { set_error("m must be < 2^32"); return SBH_EINVAL; }
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, train_carve(nullptr, m).total, &done);
    if (rc || done) return rc;
    if (m == 0 || !d_samples || !d_model) { set_error("empty sample or null pointer"); return SBH_EINVAL; }
    if (steps < 0 || batch < kBatchUnit || batch % kBatchUnit || batch > kMaxBatch) {
        set_error("batch must be a multiple of %d in [%d, %d]", kBatchUnit, kBatchUnit, kMaxBatch);
        return SBH_EINVAL;
    }
    cudaStream_t s = as_stream(stream);
    TrainScratch t = train_carve(d_scratch, m);
    Model* model = static_cast<Model*>(d_model);
    SBH_CUDA(cudaMemsetAsync(model, 0, sizeof(Model), s));
    SBH_CUDA(cudaMemsetAsync(t.bar, 0, 2 * sizeof(uint32_t), s));
    if (d_init_params)
        SBH_CUDA(cudaMemcpyAsync(t.params, d_init_params, kNP * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // sort the sample (its pointers are not needed: row numbers, made by the
    // sort's first pass)
    const unsigned gm = (unsigned)((m + 255) / 256);
    rc = sort_by_value(d_samples, nullptr, t.s_keys, t.s_ptrs, m, t.sort_scratch, s, RadixValue{}, kPositions,
                       "learned_sample");
    if (rc) return rc;
    // heavy keys (in key order, the first kMaxHeavy), the non-heavy samples,
    // training rows
    const uint32_t nb = (uint32_t)((m + kCompactTile - 1) / kCompactTile);
    const uint64_t c_min = n_rows ? (uint64_t)(SBH_LEARNED_CAPACITY / kHeavyDiv) * m / n_rows + 1 : m + 1;
    const HeavyRunStart heavy_pred{t.s_keys, m, c_min};
    SBH_TIMED("learned_heavy", s,
              compact_count_kernel<HeavyRunStart><<<nb, kCompactTile, 0, s>>>(m, heavy_pred, t.block_sums));
    SBH_LAUNCHED();
    SBH_TIMED("learned_heavy", s, scan_u64_kernel<<<1, 1024, 0, s>>>(t.block_sums, nb, &model->heavy_count));
    SBH_LAUNCHED();
    SBH_TIMED("learned_heavy", s,
              compact_scatter_kernel<HeavyRunStart><<<nb, kCompactTile, 0, s>>>(t.s_keys, m, heavy_pred, t.block_sums,
                                                                               model->heavy_keys, kMaxHeavy));
    SBH_LAUNCHED();
    const NotHeavy keep_pred{t.s_keys, model};
    SBH_TIMED("learned_keep", s, compact_count_kernel<NotHeavy><<<nb, kCompactTile, 0, s>>>(m, keep_pred, t.block_sums));
    SBH_LAUNCHED();
    SBH_TIMED("learned_keep_scan", s, scan_u64_kernel<<<1, 1024, 0, s>>>(t.block_sums, nb, t.m_train));
    SBH_LAUNCHED();
    SBH_TIMED("learned_keep", s,
              compact_scatter_kernel<NotHeavy><<<nb, kCompactTile, 0, s>>>(t.s_keys, m, keep_pred, t.block_sums, t.nh,
                                                                          m));
    SBH_LAUNCHED();
    SBH_TIMED("learned_trainset", s, trainset_kernel<<<gm, 256, 0, s>>>(t.nh, t.m_train, t.X, t.T));
    SBH_LAUNCHED();
    if (!d_init_params) {
        SBH_TIMED("learned_init", s, quantile_init_kernel<<<1, 64, 0, s>>>(t.nh, t.m_train, t.params));
        SBH_LAUNCHED();
    }
    if (d_train_x) SBH_CUDA(cudaMemcpyAsync(d_train_x, t.X, m * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (d_train_t) SBH_CUDA(cudaMemcpyAsync(d_train_t, t.T, m * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // train
    if (steps > 0) {
        TrainArgs a{t.X, t.T, t.m_train, t.params, t.partial, t.partial_sq, t.bar, d_losses,
                    steps, batch, lr, spin_limit(), status_word()};
        const size_t smem = sizeof(GradSmem);
        SBH_CUDA(cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        SBH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, train_kernel, kGThreads, smem));
        if (per_sm * num_sms() < kTrainCtas) { set_error("cannot co-schedule %d training CTAs", kTrainCtas); return SBH_ECUDA; }
        void* args[] = {&a};
        {
            ProfScope ps("learned_train", s);
            SBH_CUDA(cudaLaunchCooperativeKernel((const void*)train_kernel, dim3(kTrainCtas), dim3(kGThreads), args,
                                                 smem, s));
        }
    }
    SBH_TIMED("learned_finish", s,
              finish_model_kernel<<<1, 256, 0, s>>>(t.params, t.m_train, SBH_LEARNED_CAPACITY, model));
    SBH_LAUNCHED();
    return SBH_OK;
}

}  // extern "C"

extern "C" int sbh_kpa_sort_learned(const uint64_t* d_keys_in, const uint32_t* d_ptrs_in, uint64_t* d_keys_out,
                                    uint32_t* d_ptrs_out, uint64_t n, const void* d_model, uint64_t* d_stats,
                                    void* d_scratch, size_t* scratch_bytes, void* stream) {
    using namespace sbh;
    clear_error();
    if (n > 0xFFFFFFFFull) { set_error("n must be < 2^32"); return SBH_EINVAL; }
    bool done = false;
    int rc = scratch_check(d_scratch, scratch_bytes, learned_carve(nullptr, n).total, &done);
    if (rc || done) return rc;
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        if (d_stats) SBH_CUDA(cudaMemsetAsync(d_stats, 0, SBH_LEARNED_STATS * sizeof(uint64_t), s));
        return SBH_OK;
    }
    if (!d_keys_in || !d_keys_out || !d_ptrs_out || !d_model) { set_error("null pointer"); return SBH_EINVAL; }
    if (d_keys_in == d_keys_out) { set_error("the learned sort needs distinct input and output buffers"); return SBH_EINVAL; }
    SortLearnedScratch t = learned_carve(d_scratch, n);
    const Model* model = static_cast<const Model*>(d_model);
    SBH_CUDA(cudaMemsetAsync(t.heavy_bucket_bits, 0, t.zero_bytes, s));
    // bucket count: about two buckets per capacity; when every id can stay
    // below 2^16 with at most a quarter fewer spread buckets, the ids are
    // carried in 16 bits through two digit passes (the count and the heavy
    // keys used are settled on the device)
    const uint64_t nb_n = learned_nb(n);
    const bool carry = nb_n - nb_n / 4 <= kMaxBucketIds - 3ull;
    uint32_t* nbid = t.small + 0;
    uint32_t* counter = t.small + 1;
    uint32_t* nlist = t.small + 2;
    uint32_t* rows_total = t.small + 3;
    uint32_t* lplan = t.small + 4;  // heavy keys used, spread buckets
    SBH_TIMED("learned_plan", s, learned_plan_kernel<<<1, 32, 0, s>>>(model, (uint32_t)nb_n, carry ? 1 : 0, lplan));
    SBH_LAUNCHED();
    SBH_CUDA(cudaMemsetAsync(t.cell_hc, 0, (kNCell + 1) * sizeof(uint32_t), s));
    SBH_CUDA(cudaMemsetAsync(t.cell_hidx, 0xFF, (kNCell + 1) * sizeof(uint32_t), s));
    SBH_TIMED("learned_heavy_cells", s,
              heavy_cells_kernel<<<(kMaxHeavy + 255) / 256, 256, 0, s>>>(model, lplan, t.cell_hc, t.cell_hidx));
    SBH_LAUNCHED();
    SBH_TIMED("learned_cdf", s,
              cell_cdf_kernel<<<kTblBlocks, kTblThreads, 0, s>>>(model, t.F, t.cell_hc, t.bmax, t.bheavy));
    SBH_LAUNCHED();
    SBH_TIMED("learned_table", s,
              cell_table_kernel<<<kTblBlocks, kTblThreads, 0, s>>>(model, t.F, t.cell_hc, t.cell_hidx, t.hcells,
                                                                   t.bmax, t.bheavy, lplan + 1, t.cells, t.cells16,
                                                                   t.heavy_bucket_bits, nbid));
    SBH_LAUNCHED();
    const BucketValue fn{t.cells, t.hcells, model->heavy_keys};
    if (carry) {
        rc = sort_by_carried_ids(d_keys_in, d_ptrs_in, d_keys_out, d_ptrs_out, n, t.sort_scratch, s,
                                 BucketValue16{t.cells16, t.hcells, model->heavy_keys}, nbid, t.bstart,
                                 t.small + 12);
        if (rc) return rc;
    } else {
        // stable scatter by bucket id computed from the key (ids below 2^24)
        rc = sort_by_value(d_keys_in, d_ptrs_in, d_keys_out, d_ptrs_out, n, t.sort_scratch, s, fn, 3, "learned_ids");
        if (rc) return rc;
        SBH_TIMED("learned_bounds", s,
                  bucket_bounds_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_keys_out, (uint32_t)n, fn, nbid,
                                                                                   t.bstart));
        SBH_LAUNCHED();
    }
    // the bucket sort's runs, listed in t.list (free until the overflow list)
    const unsigned lblocks = (unsigned)(learned_max_ids(n) / 1024 + 1);
    uint32_t* nruns = t.small + 6;
    SBH_TIMED("learned_runs", s, run_start_kernel<<<lblocks, 1024, 0, s>>>(t.bstart, nbid, t.heavy_bucket_bits, t.run_flag));
    SBH_LAUNCHED();
    SBH_TIMED("learned_runs_count", s, flag_count_kernel<<<lblocks, 1024, 0, s>>>(t.run_flag, nbid, t.bstart, t.bagg));
    SBH_LAUNCHED();
    SBH_TIMED("learned_runs_list", s,
              flag_list_kernel<<<lblocks, 1024, 0, s>>>(t.run_flag, nbid, t.bstart, t.bagg, t.list, t.offs, nruns,
                                                        t.small + 7));
    SBH_LAUNCHED();
    SBH_TIMED("learned_runs_rec", s,
              run_records_kernel<<<lblocks, 1024, 0, s>>>(t.list, nruns, 0, nbid, t.bstart, t.heavy_bucket_bits,
                                                          t.runrec));
    SBH_LAUNCHED();
    const size_t smem = sizeof(BucketSmem);
    SBH_CUDA(cudaFuncSetAttribute(bucket_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SBH_TIMED("learned_bucket_sort", s,
              bucket_sort_kernel<<<num_sms(), kBThreads, smem, s>>>(d_keys_out, d_ptrs_out, t.bstart, t.runrec,
                                                                    nruns, counter, t.ov_flag, t.retry_flag,
                                                                    t.stats));
    SBH_LAUNCHED();
    // runs whose group sort failed: their buckets one by one (usually none)
    uint32_t* nretry = t.small + 9;
    SBH_TIMED("learned_retry_count", s,
              flag_count_kernel<<<lblocks, 1024, 0, s>>>(t.retry_flag, nbid, t.bstart, t.bagg));
    SBH_LAUNCHED();
    SBH_TIMED("learned_retry_list", s,
              flag_list_kernel<<<lblocks, 1024, 0, s>>>(t.retry_flag, nbid, t.bstart, t.bagg, t.list, t.offs, nretry,
                                                        t.small + 10));
    SBH_LAUNCHED();
    SBH_TIMED("learned_retry_rec", s,
              run_records_kernel<<<lblocks, 1024, 0, s>>>(t.list, nretry, 1, nbid, t.bstart, t.heavy_bucket_bits,
                                                          t.runrec));
    SBH_LAUNCHED();
    SBH_TIMED("learned_bucket_retry", s,
              bucket_sort_kernel<<<num_sms(), kBThreads, smem, s>>>(d_keys_out, d_ptrs_out, t.bstart, t.runrec,
                                                                    nretry, t.small + 8, t.ov_flag, t.retry_flag,
                                                                    t.stats));
    SBH_LAUNCHED();
    SBH_TIMED("learned_overflow_count", s,
              flag_count_kernel<<<lblocks, 1024, 0, s>>>(t.ov_flag, nbid, t.bstart, t.bagg));
    SBH_LAUNCHED();
    SBH_TIMED("learned_overflow_list", s,
              flag_list_kernel<<<lblocks, 1024, 0, s>>>(t.ov_flag, nbid, t.bstart, t.bagg, t.list, t.offs, nlist,
                                                        rows_total));
    SBH_LAUNCHED();
    // the overflow rows (their number is known only on the device): gathered
    // into a compact buffer, sorted by the plain radix sort sized on the
    // device, and put back
    const unsigned mg = (unsigned)min_u64((n + 255) / 256, (uint64_t)num_sms() * 8);
    SBH_TIMED("learned_overflow_move", s,
              overflow_move_kernel<<<mg, 256, 0, s>>>(d_keys_out, d_ptrs_out, t.bstart, t.list, t.offs, nlist,
                                                      rows_total, t.ck, t.cp, 1));
    SBH_LAUNCHED();
    rc = sort_by_value(t.ck, t.cp, t.ck, t.cp, n, t.sort_scratch, s, RadixValue{}, kPositions, "learned_overflow",
                       rows_total);
    if (rc) return rc;
    SBH_TIMED("learned_overflow_move", s,
              overflow_move_kernel<<<mg, 256, 0, s>>>(d_keys_out, d_ptrs_out, t.bstart, t.list, t.offs, nlist,
                                                      rows_total, t.ck, t.cp, 0));
    SBH_LAUNCHED();
    if (d_stats) {
        SBH_TIMED("learned_stats", s, learned_stats_kernel<<<1, 1024, 0, s>>>(nbid, lplan, t.bstart, t.stats, t.small + 12, d_stats));
        SBH_LAUNCHED();
    }
    return SBH_OK;
}
