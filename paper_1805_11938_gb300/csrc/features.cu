// Matrix features (Sec. V-B "Features", Table IV), their scaling (Sec. V-B
// "Feature Scaling") and the selector network (Sec. V-A/V-B: features in,
// representation label out; here a 16-64-64-5 multilayer perceptron, one of
// the alternatives of Sec. V-D), with its training kernels.
//
// Feature definitions (len_i = ptr[i+1] - ptr[i]; the row-length statistics
// are exact over all M rows, the histogram and index statistics come from a
// row sample R = all rows, or rows floor(k*M/8192) for k < 8192):
//   0 n_rows  1 n_cols  2 nnz/(M*N)  3 min len  4 max len  5 mean = nnz/M
//   6 std of len  7 std/mean  8 log2(max(nnz,1))  9 mean/max
//  10 HYB tail fraction over R with K from R (lengths capped at 512)
//  11 mean |col-row| and 12 max |col-row| over the first 16 entries of each sampled row
//  13 fraction of empty rows  14 fraction of rows with len >= 32
//  15 SELL-32 fill over R sorted, lengths capped at 512
//
// Two launches.  k_rowstats reads ptr once with the whole GPU and reduces the
// exact statistics (min, max, sum of squares, empty rows, rows of length >= 32)
// into one slot of a small static device array (each block adds its totals
// with relaxed atomics and exits).  The features kernel, launched behind it with
// programmatic stream serialization, is one thread-block cluster (16 CTAs x
// 512 threads where the device can place one, else 8 x 1024), one sampled row
// per thread.  Each CTA reduces its rows, then adds its statistics and its
// length histogram into CTA 0's shared memory with cluster shared-memory
// atomics; after one cluster barrier two warps of CTA 0 wait for k_rowstats
// and finish: warp 1 scans the histogram while warp 0 evaluates the features
// as straight-line code, then, for a selection, both run the network.  A lone
// warp's dependent instructions are the cost there, so that code avoids
// divergent per-feature branches and keeps its divisions independent.
//
// Selection never returns ELL when its padded layout (ceil(M/4)*4 rows of
// max-len slots, 12 bytes each, plus the row lengths) would exceed the
// model's max_bytes: the exact longest row makes that footprint exact, and
// the argmax is then taken over the other four formats.  The other layouts
// stay within a small multiple of the CSR (SELL: nnz + C * max-len slots;
// HYB: K * M <= 3 * nnz slots by the rule for K; CSR5: the CSR padded to
// whole tiles).
#include <atomic>
#include <mutex>
#include <cooperative_groups.h>
#include <cuda_pipeline.h>

#include "internal.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

struct spmv_model {
    float* params = nullptr;  // SPMV_MLP_PARAMS
    float* lo = nullptr;      // 16
    float* hi = nullptr;      // 16
    int64_t max_bytes = 0;    // selection refuses ELL layouts larger than this
};

namespace spmv {

constexpr int kFeatCtasSmall = 8;   // CTAs of the features cluster: the portable size
constexpr int kFeatCtasLarge = 16;  // and the largest, where the device allows it
constexpr int kSample = 8192;       // sampled rows: one per thread of the cluster
constexpr int kLenCap = 512;
constexpr int kSpread = 16;

// parameter offsets inside the flat vector
constexpr int oW1 = 0, oB1 = 1024, oW2 = 1088, oB2 = 5184, oW3 = 5248, oB3 = 5568, kNP = 5573;

// Transform and min-max scaling of one feature.  FP32 on purpose: this GPU's
// FP64 pipe makes double log2/division/sqrt several microseconds slower, and
// the features are float32 values to begin with.  Both logarithms are taken
// and one is selected, so lanes scaling different features do not diverge.
// The scaling's quotient uses the two-ulp division (reciprocal and multiply,
// no branch to a slow path); its operands lie far inside that division's
// range.  The features themselves keep correctly rounded divisions.
__device__ __forceinline__ float feat_transform(int j, float f) {
    constexpr unsigned kLog1p = (1u << 0) | (1u << 1) | (1u << 3) | (1u << 4) | (1u << 5) | (1u << 6) | (1u << 11) |
                                (1u << 12);
    const float a = log2f(1.0f + f);
    const float b = -log2f(fmaxf(f, 0x1.0p-60f));
    return ((kLog1p >> j) & 1u) ? a : (j == 2 ? b : f);
}

__device__ __forceinline__ float feat_scale(int j, float f, const float* lo, const float* hi) {
    const float t = feat_transform(j, f);
    const float span = hi[j] - lo[j];
    const float x = __fdividef(t - lo[j], span);
    return !(span > 0.0f) ? 0.0f : (x < 0.0f ? 0.0f : (x > 1.0f ? 1.0f : x));
}

// Barrier of the first two warps only (named barrier 1), for the tail of the
// features kernel that runs in warps 0 and 1 after the others have left.
__device__ __forceinline__ void tail_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// The cluster barrier in its two halves: arrive releases this thread's earlier
// shared-memory writes to the cluster, wait acquires everyone's.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(dev::kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned warp_sum_u32(unsigned v) { return __reduce_add_sync(dev::kFull, v); }
__device__ __forceinline__ int warp_min_i32(int v) { return __reduce_min_sync(dev::kFull, v); }
__device__ __forceinline__ int warp_max_i32(int v) { return __reduce_max_sync(dev::kFull, v); }
__device__ __forceinline__ float u64_to_f32(unsigned long long v) { return (float)v; }

// 16 -> 64 -> 64 -> 5 forward for one sample in threads 0..63 (warps 0 and
// 1), th in shared memory, xs the 16 scaled features.  Hidden unit j of each
// layer is thread j's dot product, split over independent accumulators so the
// FMA chains stay short (consecutive j: conflict-free weight reads; the inputs
// are broadcast).  Warp 0 alone computes the five outputs, four lanes each
// (output c in lanes 4c..4c+3), writes them to z_out if given, and returns in
// every lane the index of the largest (the first of equal maxima; ELL only
// when ell_ok).  Warp 1 returns -1 once the second layer is done.
__device__ int mlp_forward_64(const float* th, const float* xs, float* h1, float* h2, float* z_out, bool ell_ok = true) {
    const int j = threadIdx.x;
    float a0 = th[oB1 + j], a1 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
        a0 = fmaf(xs[i], th[oW1 + i * 64 + j], a0);
        a1 = fmaf(xs[i + 1], th[oW1 + (i + 1) * 64 + j], a1);
    }
    a0 += a1;
    h1[j] = a0 > 0.f ? a0 : 0.f;
    tail_sync();
    float c0 = th[oB2 + j], c1 = 0.f, c2 = 0.f, c3 = 0.f;
    const float4* h14 = reinterpret_cast<const float4*>(h1);
#pragma unroll
    for (int i = 0; i < 64; i += 4) {
        const float4 v = h14[i / 4];
        c0 = fmaf(v.x, th[oW2 + i * 64 + j], c0);
        c1 = fmaf(v.y, th[oW2 + (i + 1) * 64 + j], c1);
        c2 = fmaf(v.z, th[oW2 + (i + 2) * 64 + j], c2);
        c3 = fmaf(v.w, th[oW2 + (i + 3) * 64 + j], c3);
    }
    c0 = (c0 + c1) + (c2 + c3);
    h2[j] = c0 > 0.f ? c0 : 0.f;
    tail_sync();
    if (j >= 32) return -1;
    // lane 4c + p sums inputs p, p + 4, ..., p + 60 of output c (conflict-free reads)
    const int c = j >> 2, part = j & 3, cc = c < 5 ? c : 0;
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int t = 0; t < 16; t += 2) {
        d0 = fmaf(h2[part + 4 * t], th[oW3 + (part + 4 * t) * 5 + cc], d0);
        d1 = fmaf(h2[part + 4 * (t + 1)], th[oW3 + (part + 4 * (t + 1)) * 5 + cc], d1);
    }
    float zc = d0 + d1;
    zc += __shfl_xor_sync(dev::kFull, zc, 1);
    zc += __shfl_xor_sync(dev::kFull, zc, 2);
    zc += th[oB3 + cc];
    if (z_out && part == 0 && c < 5) z_out[c] = zc;
    float best = __shfl_sync(dev::kFull, zc, 0);
    int bi = 0;
#pragma unroll
    for (int q = 1; q < 5; ++q) {
        const float v = __shfl_sync(dev::kFull, zc, 4 * q);
        if (v > best && (q != SPMV_ELL || ell_ok)) {
            best = v;
            bi = q;
        }
    }
    return bi;
}

// ------------------------------------------------------- exact row lengths
//
// One slot of the ring holds one call's accumulators.  The features kernel
// reads them once k_rowstats has completed and sets them back to zero, so
// every call finds its slot at zero.  Calls take slots in turn on the host, so
// up to kRowSlots calls may be in flight on one device at once; a CUDA graph
// replays the slot it captured.  The minimum is accumulated as the maximum of
// ~len, so that zero is the identity of every accumulator.
struct __align__(32) RowStatsSlot {
    unsigned long long acc_sq;
    unsigned acc_max, acc_cmin, acc_empty, acc_long;
};
constexpr int kRowSlots = 64;
static __device__ RowStatsSlot g_rowstats[kRowSlots];

constexpr int kRowStatsThreads = 256;
constexpr int kRowStatsUnroll = 4;  // 16-byte loads in flight per thread

template <bool VEC>
__global__ void __launch_bounds__(kRowStatsThreads, 6) k_rowstats(const int32_t* __restrict__ ptr, int32_t m,
                                                               RowStatsSlot* __restrict__ slot) {
    dev::pdl_trigger();  // the features kernel behind this one may start now
    unsigned mx = 0, cmn = 0, emp = 0, lng = 0;
    unsigned long long sq = 0;
    auto add = [&](int32_t len) {
        const unsigned l = (unsigned)len;
        mx = max(mx, l);
        cmn = max(cmn, ~l);
        sq += (unsigned long long)l * l;
        emp += l == 0u;
        lng += l >= 32u;
    };
    const int lane = threadIdx.x & 31;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    int64_t tail0 = 0;
    if constexpr (VEC) {
        // quad q = rows 4q .. 4q+3 from one 16-byte load of ptr[4q .. 4q+3];
        // ptr[4q+4] is the next lane's first word (loaded directly by lane 31
        // and by the last quad).  A warp takes kRowStatsUnroll runs of 32
        // consecutive quads at a time, all loads issued before any is used.
        const int64_t nq = (int64_t)m / 4;
        constexpr int U = kRowStatsUnroll;
        for (int64_t qb = (gt - lane) * U; qb < nq; qb += nt * U) {  // warp-uniform bound
            int4 v[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int64_t q = qb + 32 * k + lane;
                v[k] = q < nq ? __ldcs(reinterpret_cast<const int4*>(ptr) + q) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int64_t q = qb + 32 * k + lane;
                int32_t nx = __shfl_down_sync(dev::kFull, v[k].x, 1);
                if (q < nq) {
                    if (lane == 31 || q + 1 == nq) nx = __ldcs(ptr + 4 * q + 4);
                    add(v[k].y - v[k].x);
                    add(v[k].z - v[k].y);
                    add(v[k].w - v[k].z);
                    add(nx - v[k].w);
                }
            }
        }
        tail0 = 4 * nq;
    }
    for (int64_t r = tail0 + gt; r < m; r += nt) add(__ldcs(ptr + r + 1) - __ldcs(ptr + r));
    mx = __reduce_max_sync(dev::kFull, mx);
    cmn = __reduce_max_sync(dev::kFull, cmn);
    emp = __reduce_add_sync(dev::kFull, emp);
    lng = __reduce_add_sync(dev::kFull, lng);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(dev::kFull, sq, o);
    __shared__ unsigned red[kRowStatsThreads / 32][4];
    __shared__ unsigned long long red_sq[kRowStatsThreads / 32];
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        red[w][0] = mx;
        red[w][1] = cmn;
        red[w][2] = emp;
        red[w][3] = lng;
        red_sq[w] = sq;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 1; i < kRowStatsThreads / 32; ++i) {
        mx = max(mx, red[i][0]);
        cmn = max(cmn, red[i][1]);
        emp += red[i][2];
        lng += red[i][3];
        sq += red_sq[i];
    }
    {
        using ref_u = cuda::atomic_ref<unsigned, cuda::thread_scope_device>;
        using ref_ull = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;
        ref_u(slot->acc_max).fetch_max(mx, cuda::memory_order_relaxed);
        ref_u(slot->acc_cmin).fetch_max(cmn, cuda::memory_order_relaxed);
        ref_u(slot->acc_empty).fetch_add(emp, cuda::memory_order_relaxed);
        ref_u(slot->acc_long).fetch_add(lng, cuda::memory_order_relaxed);
        ref_ull(slot->acc_sq).fetch_add(sq, cuda::memory_order_relaxed);
    }
}

// The features kernel: one cluster of CTAS CTAs, kSample / CTAS threads each,
// one sampled row per thread.  VEC: idx is 16-byte aligned and each sampled
// row's first entries are read as the aligned 16-byte words covering them
// (at most five), else one 4-byte load each (at most sixteen).
template <int CTAS, bool VEC>
__global__ void __launch_bounds__(kSample / CTAS)
    k_features(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, int32_t m, int32_t n, int64_t nnz,
               RowStatsSlot* __restrict__ rs, float* __restrict__ feat_out,
               const float* __restrict__ model_params, const float* __restrict__ lo, const float* __restrict__ hi,
               int64_t ell_cap, int32_t* __restrict__ fmt_out, float* __restrict__ logits_out) {
    constexpr int T = kSample / CTAS;
    constexpr int NW = T / 32;
    static_assert(kSample == 1 << 13 && T * CTAS == kSample && NW <= 32 && T >= 64, "sample layout");
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    // In CTA 0 these end as the cluster's totals over the sampled rows: the
    // length histogram (lengths capped at 512), sum of len and of |col - row|
    // over the first 16 entries; max |col - row|; entries in the spread sums.
    __shared__ unsigned hist[kLenCap + 1];
    __shared__ unsigned long long tot_u[2];
    __shared__ int tot_band;
    __shared__ unsigned tot_cnt;
    __shared__ unsigned long long red_u[NW][2];
    __shared__ unsigned red_c[NW][2];
    __shared__ float qop[4];
    __shared__ __align__(16) float wsm[kNP + 3 + 32];
    __shared__ int32_t nnz_sm;
    __shared__ __align__(16) float xs[16], h1[64], h2[64];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    dev::pdl_trigger();  // a product launched behind this kernel may get resident now
    // CTA 0 starts copying what its tail needs into shared memory now
    // (asynchronous copies, waited for just before the tail): nnz = ptr[m]
    // and, for a selection, the network and the scaling table.
    if (rank == 0) {
        if (tid == 0) __pipeline_memcpy_async(&nnz_sm, ptr + m, 4);
        if (model_params) {
            for (int c = tid; c < kNP / 4; c += T) __pipeline_memcpy_async(wsm + 4 * c, model_params + 4 * c, 16);
            if (tid < kNP % 4) __pipeline_memcpy_async(wsm + (kNP / 4) * 4 + tid, model_params + (kNP / 4) * 4 + tid, 4);
            if (tid < 4) __pipeline_memcpy_async(wsm + kNP + 3 + 4 * tid, lo + 4 * tid, 16);
            else if (tid < 8) __pipeline_memcpy_async(wsm + kNP + 3 + 16 + 4 * (tid - 4), hi + 4 * (tid - 4), 16);
        }
        __pipeline_commit();
    }
    for (int b = tid; b <= kLenCap; b += T) hist[b] = 0;
    if (tid < 2) tot_u[tid] = 0;
    if (tid == 0) {
        tot_band = 0;
        tot_cnt = 0;
    }
    __syncthreads();
    cluster_arrive();  // waited for before the CTAs add into CTA 0's totals

    // ---- phase 1: one sampled row per thread.  Row of sample k: k*M/S, with
    // S = 8192 = 2^13 whenever M > S (a shift), else k.
    const int64_t S = m < kSample ? m : kSample;
    const int64_t k = (int64_t)rank * T + tid;
    const bool on = k < S;
    const int32_t i = (int32_t)(m > kSample ? ((k * (int64_t)m) >> 13) : k);
    const int32_t p0 = on ? ptr[i] : 0;
    const int32_t len = on ? ptr[i + 1] - p0 : 0;
    const int ne = len < kSpread ? len : kSpread;
    unsigned long long ssum = 0;
    int band = 0;
    if constexpr (VEC) {
        const int32_t base = p0 & ~3;
        const int off = p0 - base, nv = (off + ne + 3) >> 2;
        int32_t w[4 * 5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const int64_t e0 = (int64_t)base + 4 * v;
            w[4 * v] = w[4 * v + 1] = w[4 * v + 2] = w[4 * v + 3] = i;
            if (v < nv) {  // the word holds entries of the window
                if (e0 + 4 <= nnz) {
                    const int4 t = __ldg(reinterpret_cast<const int4*>(idx + e0));
                    w[4 * v] = t.x;
                    w[4 * v + 1] = t.y;
                    w[4 * v + 2] = t.z;
                    w[4 * v + 3] = t.w;
                } else {  // the end of idx: the row's own entries one by one
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (e0 + u < p0 + ne) w[4 * v + u] = __ldg(idx + e0 + u);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 4 * 5; ++t) {
            const int d = w[t] - i;
            const int ad = (t >= off && t < off + ne) ? (d < 0 ? -d : d) : 0;
            ssum += (unsigned)ad;
            band = max(band, ad);
        }
    } else {
        int32_t w[kSpread];
#pragma unroll
        for (int q = 0; q < kSpread; ++q) w[q] = q < ne ? __ldg(idx + p0 + q) : i;
#pragma unroll
        for (int q = 0; q < kSpread; ++q) {
            const int d = w[q] - i;
            const int ad = d < 0 ? -d : d;
            ssum += (unsigned)ad;
            band = max(band, ad);
        }
    }
    {  // one shared atomic per distinct bin in the warp
        const unsigned act = __ballot_sync(dev::kFull, on);
        if (on) {
            const int bin = len < 0 ? 0 : (len < kLenCap ? len : kLenCap);  // in range even for a malformed ptr
            const unsigned peers = __match_any_sync(act, bin);
            if (lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
        }
    }
    {
        const unsigned long long a0 = warp_sum_u64(on ? (unsigned long long)len : 0ull);
        const unsigned long long a2 = warp_sum_u64(ssum);
        const int i2 = warp_max_i32(band);
        const unsigned c2 = warp_sum_u32((unsigned)ne);
        if (lane == 0) {
            red_u[warp][0] = a0;
            red_u[warp][1] = a2;
            red_c[warp][0] = (unsigned)i2;
            red_c[warp][1] = c2;
        }
    }
    __syncthreads();
    // Every CTA's totals and histogram have been initialised: add this CTA's
    // statistics and nonzero histogram bins into CTA 0's (cluster shared-memory
    // atomics, one statistic per lane); one cluster barrier publishes them.
    cluster_wait();
    if (rank != 0) {
        unsigned* h0 = cluster.map_shared_rank(hist, 0);
        for (int b = tid; b <= kLenCap; b += T) {
            const unsigned v = hist[b];
            if (v) atomicAdd(h0 + b, v);
        }
    }
    if (warp == 0) {
        const bool ok = lane < NW;
        const unsigned long long a0 = warp_sum_u64(ok ? red_u[lane][0] : 0ull);
        const unsigned long long a2 = warp_sum_u64(ok ? red_u[lane][1] : 0ull);
        const int i2 = warp_max_i32(ok ? (int)red_c[lane][0] : 0);
        const unsigned c2 = warp_sum_u32(ok ? red_c[lane][1] : 0u);
        unsigned long long* tu = cluster.map_shared_rank(tot_u, 0);
        if (lane < 2) atomicAdd(tu + lane, lane == 0 ? a0 : a2);
        else if (lane == 2) atomicMax(cluster.map_shared_rank(&tot_band, 0), i2);
        else if (lane == 3) atomicAdd(cluster.map_shared_rank(&tot_cnt, 0), c2);
    }
    cluster.sync();
    if (rank != 0) return;  // CTA 0 holds everything now
    __pipeline_wait_prior(0);
    __syncthreads();  // every thread's copies (nnz, the network, the scaling table) have landed
    if (tid >= 64) return;

    // ---- phase 2 (CTA 0, warps 0 and 1): warp 1 scans the histogram while
    // warp 0 computes the features that do not need it; then warp 0 finishes
    // the features and, for a selection, both warps run the network.
    const unsigned cnt = (unsigned)S;
    if (warp == 1) {
        // c_b = #{len >= b} over the capped histogram: suffix sums, lane l
        // owning bins 17l .. 17l + 16 (in-lane, then over the lanes).  c_b is
        // non-increasing, so the bins with c_b >= ceil(S/3) are 1..K of the
        // HYB rule and the K-dependent sum needs no second pass.
        constexpr int PB = 17;  // 32 * 17 = 544 >= 513
        unsigned cb[PB];
        unsigned run = 0;
#pragma unroll
        for (int q = PB - 1; q >= 0; --q) {
            const int bb = lane * PB + q;
            run += bb <= kLenCap ? hist[bb] : 0u;
            cb[q] = run;
        }
        unsigned later = run;  // this lane's total, then the totals of later lanes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_down_sync(dev::kFull, later, d);
            if (lane + d < 32) later += u;
        }
        later -= run;
        const unsigned need = (cnt + 2) / 3;
        unsigned wpart = 0, cpart = 0, upart = 0;
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int bb = lane * PB + q;
            const unsigned v = cb[q] + later;
            if (bb >= 1 && bb <= kLenCap) {
                wpart += (v + 31) >> 5;
                cpart += v;
                upart += v >= need ? v : 0u;
            }
        }
        const unsigned widths = warp_sum_u32(wpart);      // SELL-32 slice widths
        const unsigned capped_sum = warp_sum_u32(cpart);  // sum of min(len, 512)
        const unsigned upto_k = warp_sum_u32(upart);      // sum of min(len, K)
        // the operands of the two quotients that need the scans (features 10, 15)
        const unsigned long long sum_len = tot_u[0];
        if (lane == 0) {
            qop[0] = sum_len > 0 ? u64_to_f32(sum_len - upto_k) : 0.0f;
            qop[1] = sum_len > 0 ? u64_to_f32(sum_len) : 1.0f;
            qop[2] = widths > 0 ? (float)capped_sum : 1.0f;
            qop[3] = widths > 0 ? 32.0f * (float)widths : 1.0f;
        }
    }
    // Warp 0: the features as straight-line code, the same in every lane
    // (FP32 throughout, exact integer parts in 64 bits), except that each lane
    // takes the one quotient of its own feature, so the correctly rounded
    // divisions run side by side rather than one after another.
    float f = 0.0f;
    bool ell_ok = true;
    if (warp == 0) {
        dev::pdl_wait();  // k_rowstats has completed: its totals are visible
        const int j = lane & 15;
        const unsigned long long spread_sum = tot_u[1];
        const unsigned long long sum_len = (unsigned long long)(unsigned)nnz_sm;  // exact, all rows
        const unsigned long long sum_sq = rs->acc_sq;
        const int min_len = (int)~rs->acc_cmin, max_len = (int)rs->acc_max, bandw = tot_band;
        const unsigned empty = rs->acc_empty, longc = rs->acc_long, spread_cnt = tot_cnt;
        __syncwarp();
        if (lane == 0) {  // the slot starts the next call that takes it at zero
            rs->acc_sq = 0ull;
            rs->acc_max = rs->acc_cmin = rs->acc_empty = rs->acc_long = 0u;
        }
        const unsigned rows = (unsigned)m;
        const float fc = (float)m;
        const float nz = (float)nnz_sm;
        const float mean = nz / fc;
        // std = sqrt(M * sum_sq - nnz^2) / M, the difference in exact 128-bit integer arithmetic
        const unsigned long long a_lo = (unsigned long long)rows * sum_sq;
        const unsigned long long a_hi = __umul64hi((unsigned long long)rows, sum_sq);
        const unsigned long long b_lo = sum_len * sum_len;
        const unsigned long long b_hi = __umul64hi(sum_len, sum_len);
        const unsigned long long d_lo = a_lo - b_lo;
        const unsigned long long d_hi = a_hi - b_hi - (a_lo < b_lo ? 1ull : 0ull);
        const float sd = sqrtf(u64_to_f32(d_hi) * 18446744073709551616.0f + u64_to_f32(d_lo)) / fc;
        const float spread = u64_to_f32(spread_sum), spread_n = (float)spread_cnt;
        // the ELL layout's footprint, exact from the longest row
        const long long ld = ((long long)m + 3) / 4 * 4;
        ell_ok = ld * (long long)max_len * 12 + ld * 4 <= (long long)ell_cap;
        const float lg = log2f(nnz_sm > 1 ? nz : 1.0f);
        // numerator and denominator of this lane's quotient (0 / 1 where it has none)
        float num = 0.0f, den = 1.0f;
        num = j == 2 || j == 5 ? nz : num;
        den = j == 2 ? (float)m * (float)n : den;
        den = j == 5 ? (float)m : den;
        num = j == 7 ? (sum_len > 0 ? sd : 0.0f) : num;
        den = j == 7 ? (sum_len > 0 ? mean : 1.0f) : den;
        num = j == 9 ? (max_len > 0 ? mean : 0.0f) : num;
        den = j == 9 ? (max_len > 0 ? (float)max_len : 1.0f) : den;
        num = j == 11 ? (spread_cnt > 0 ? spread : 0.0f) : num;
        den = j == 11 ? (spread_cnt > 0 ? spread_n : 1.0f) : den;
        num = j == 13 ? (float)empty : num;
        num = j == 14 ? (float)longc : num;
        den = j == 13 || j == 14 ? fc : den;
        tail_sync();  // the scans' operands are in qop
        num = j == 10 ? qop[0] : num;
        den = j == 10 ? qop[1] : den;
        num = j == 15 ? qop[2] : num;
        den = j == 15 ? qop[3] : den;
        f = num / den;
        f = j == 0 ? (float)m : f;
        f = j == 1 ? (float)n : f;
        f = j == 3 ? (float)min_len : f;
        f = j == 4 ? (float)max_len : f;
        f = j == 6 ? sd : f;
        f = j == 8 ? lg : f;
        f = j == 12 ? (float)bandw : f;
        if (lane < 16) {
            if (feat_out) feat_out[lane] = f;
            if (model_params) xs[lane] = feat_scale(lane, f, wsm + kNP + 3, wsm + kNP + 3 + 16);
        }
    } else {
        tail_sync();
    }
    if (!model_params) return;
    tail_sync();
    const int best = mlp_forward_64(wsm, xs, h1, h2, logits_out, ell_ok);
    if (tid == 0 && fmt_out) fmt_out[0] = best;
}

// The features kernel, launched behind k_rowstats with programmatic stream
// serialization (its sampled part overlaps the exact pass over ptr).
template <int CTAS, bool VEC>
static cudaError_t launch_features_k(const spmv_csr* c, RowStatsSlot* rs, float* feat, const spmv_model* model,
                                     int32_t* fmt, float* logits, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CTAS, 1, 1);
    cfg.blockDim = dim3(kSample / CTAS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CTAS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_features<CTAS, VEC>, c->ptr, c->idx, c->m, c->n, (int64_t)c->nnz, rs, feat,
                              model ? (const float*)model->params : nullptr, model ? (const float*)model->lo : nullptr,
                              model ? (const float*)model->hi : nullptr, model ? model->max_bytes : (int64_t)0, fmt,
                              logits);
}

// This device's ring of row-statistics slots (looked up once per device, with
// that device current) and the next slot in turn.
static int rowstats_slot(RowStatsSlot** out) {
    static std::mutex mu;
    static RowStatsSlot* base[64] = {};
    static std::atomic<unsigned> next{0};
    int dev = 0;
    SPMV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(SPMV_ERR_INVALID_ARG, "device %d out of range", dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!base[dev]) {
            void* p = nullptr;
            SPMV_CUDA(cudaGetSymbolAddress(&p, g_rowstats));
            base[dev] = static_cast<RowStatsSlot*>(p);
        }
    }
    *out = base[dev] + (next.fetch_add(1u, std::memory_order_relaxed) % kRowSlots);
    return SPMV_OK;
}

static cudaError_t launch_rowstats(const spmv_csr* c, RowStatsSlot* rs, cudaStream_t s) {
    const bool vec = (reinterpret_cast<uintptr_t>(c->ptr) & 15) == 0;
    const int64_t items = vec ? (int64_t)c->m / 4 / kRowStatsUnroll : (int64_t)c->m;
    const int g = grid_capped(items > 0 ? items : 1, kRowStatsThreads, 6);
    if (vec) k_rowstats<true><<<g, kRowStatsThreads, 0, s>>>(c->ptr, c->m, rs);
    else k_rowstats<false><<<g, kRowStatsThreads, 0, s>>>(c->ptr, c->m, rs);
    return cudaGetLastError();
}

// The cluster size for this device: 16 CTAs (a non-portable size, opted into
// here) where one such cluster can be resident, else the portable 8.  Both
// give the same features bit for bit (exact integer statistics, the same FP32
// code after them).  Cached per device.
static std::atomic<int> g_force_ctas{0};

static int features_ctas() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kFeatCtasSmall;
    const int forced = g_force_ctas.load();
    if (cached[dev]) return forced ? forced : cached[dev];
    int ctas = kFeatCtasSmall;
    if (cudaFuncSetAttribute(k_features<kFeatCtasLarge, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_features<kFeatCtasLarge, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kFeatCtasLarge, 1, 1);
        cfg.blockDim = dim3(kSample / kFeatCtasLarge, 1, 1);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kFeatCtasLarge;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_features<kFeatCtasLarge, true>, &cfg) == cudaSuccess &&
            clusters >= 1)
            ctas = kFeatCtasLarge;
    }
    (void)cudaGetLastError();  // a refused opt-in leaves the portable size
    cached[dev] = ctas;
    return forced ? forced : ctas;
}

void debug_features_cluster(int ctas) {
    g_force_ctas.store(ctas == kFeatCtasSmall || ctas == kFeatCtasLarge ? ctas : 0);
}

static int launch_features(const spmv_csr* c, float* feat, const spmv_model* model, int32_t* fmt, float* logits,
                           cudaStream_t s) {
    if (!c) return set_error(SPMV_ERR_INVALID_ARG, "csr is NULL");
    if (c->m <= 0 || c->n <= 0 || !c->ptr || (c->nnz > 0 && !c->idx) || c->nnz < 0)
        return set_error(SPMV_ERR_INVALID_ARG, "malformed csr argument");
    const bool vec = (reinterpret_cast<uintptr_t>(c->idx) & 15) == 0;
    const bool large = features_ctas() == kFeatCtasLarge;
    RowStatsSlot* rs = nullptr;
    SPMV_TRY(rowstats_slot(&rs));
    SPMV_CUDA(launch_rowstats(c, rs, s));
    const cudaError_t e = large ? (vec ? launch_features_k<kFeatCtasLarge, true>(c, rs, feat, model, fmt, logits, s)
                                       : launch_features_k<kFeatCtasLarge, false>(c, rs, feat, model, fmt, logits, s))
                                : (vec ? launch_features_k<kFeatCtasSmall, true>(c, rs, feat, model, fmt, logits, s)
                                       : launch_features_k<kFeatCtasSmall, false>(c, rs, feat, model, fmt, logits, s));
    if (e != cudaSuccess) {
        // the features kernel zeroes the slot after reading it; without it, zero it here
        (void)cudaGetLastError();
        (void)cudaMemsetAsync(rs, 0, sizeof(RowStatsSlot), s);
        return cuda_error(e, "the features kernel's launch");
    }
    return SPMV_OK;
}

// ----------------------------------------------------------------- training
//
// One CTA of 1024 threads; samples are processed in chunks of 64 with all
// activations in shared memory.  Every gradient entry is accumulated by one
// thread in a fixed order, so results are deterministic.

constexpr int kChunk = 64;

struct TrainSmem {
    float th[kNP];
    float g[kNP];
    float xb[kChunk * 16];
    float h1[kChunk * 64];
    float h2[kChunk * 64];
    float d2[kChunk * 64];  // dL/da2
    float d1[kChunk * 64];  // dL/da1
    float dz[kChunk * 5];
    float lossb[kChunk];
    float loss;
};

// grad of the mean cross-entropy over B samples into S.g; S.th holds the parameters.
__device__ void mlp_grad_block(TrainSmem& S, const float* __restrict__ X, const int32_t* __restrict__ lab, int32_t B) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int p = tid; p < kNP; p += nt) S.g[p] = 0.f;
    if (tid == 0) S.loss = 0.f;
    __syncthreads();
    const float invB = 1.0f / (float)B;
    for (int b0 = 0; b0 < B; b0 += kChunk) {
        const int nb = B - b0 < kChunk ? B - b0 : kChunk;
        for (int q = tid; q < kChunk * 16; q += nt) S.xb[q] = (q / 16 < nb) ? X[(int64_t)b0 * 16 + q] : 0.f;
        __syncthreads();
        for (int q = tid; q < kChunk * 64; q += nt) {
            const int b = q / 64, j = q % 64;
            float a = S.th[oB1 + j];
            for (int i = 0; i < 16; ++i) a = fmaf(S.xb[b * 16 + i], S.th[oW1 + i * 64 + j], a);
            S.h1[q] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        for (int q = tid; q < kChunk * 64; q += nt) {
            const int b = q / 64, j = q % 64;
            float a = S.th[oB2 + j];
            for (int i = 0; i < 64; ++i) a = fmaf(S.h1[b * 64 + i], S.th[oW2 + i * 64 + j], a);
            S.h2[q] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        if (tid < kChunk) {
            const int b = tid;
            if (b < nb) {
                float zz[5];
                float mxz = -3.4e38f;
                for (int c = 0; c < 5; ++c) {
                    float a = S.th[oB3 + c];
                    for (int i = 0; i < 64; ++i) a = fmaf(S.h2[b * 64 + i], S.th[oW3 + i * 5 + c], a);
                    zz[c] = a;
                    mxz = fmaxf(mxz, a);
                }
                float den = 0.f;
                for (int c = 0; c < 5; ++c) den += expf(zz[c] - mxz);
                const int y = lab[b0 + b];
                S.lossb[b] = -(zz[y] - mxz - logf(den));
                for (int c = 0; c < 5; ++c) S.dz[b * 5 + c] = (expf(zz[c] - mxz) / den - (c == y ? 1.f : 0.f)) * invB;
            } else {
                S.lossb[b] = 0.f;
                for (int c = 0; c < 5; ++c) S.dz[b * 5 + c] = 0.f;
            }
        }
        __syncthreads();
        if (tid == 0) {
            float l = S.loss;
            for (int b = 0; b < nb; ++b) l += S.lossb[b];
            S.loss = l;
        }
        // W3, b3
        for (int q = tid; q < 64 * 5 + 5; q += nt) {
            if (q < 320) {
                const int i = q / 5, c = q % 5;
                float a = 0.f;
                for (int b = 0; b < nb; ++b) a = fmaf(S.h2[b * 64 + i], S.dz[b * 5 + c], a);
                S.g[oW3 + q] += a;
            } else {
                const int c = q - 320;
                float a = 0.f;
                for (int b = 0; b < nb; ++b) a += S.dz[b * 5 + c];
                S.g[oB3 + c] += a;
            }
        }
        // dL/da2
        for (int q = tid; q < kChunk * 64; q += nt) {
            const int b = q / 64, i = q % 64;
            float a = 0.f;
            for (int c = 0; c < 5; ++c) a = fmaf(S.dz[b * 5 + c], S.th[oW3 + i * 5 + c], a);
            S.d2[q] = S.h2[q] > 0.f ? a : 0.f;
        }
        __syncthreads();
        // W2, b2
        for (int q = tid; q < 64 * 64 + 64; q += nt) {
            if (q < 4096) {
                const int i = q / 64, j = q % 64;
                float a = 0.f;
                for (int b = 0; b < nb; ++b) a = fmaf(S.h1[b * 64 + i], S.d2[b * 64 + j], a);
                S.g[oW2 + q] += a;
            } else {
                const int j = q - 4096;
                float a = 0.f;
                for (int b = 0; b < nb; ++b) a += S.d2[b * 64 + j];
                S.g[oB2 + j] += a;
            }
        }
        // dL/da1
        for (int q = tid; q < kChunk * 64; q += nt) {
            const int b = q / 64, i = q % 64;
            float a = 0.f;
            for (int j = 0; j < 64; ++j) a = fmaf(S.d2[b * 64 + j], S.th[oW2 + i * 64 + j], a);
            S.d1[q] = S.h1[q] > 0.f ? a : 0.f;
        }
        __syncthreads();
        // W1, b1
        for (int q = tid; q < 16 * 64 + 64; q += nt) {
            if (q < 1024) {
                const int i = q / 64, j = q % 64;
                float a = 0.f;
                for (int b = 0; b < nb; ++b) a = fmaf(S.xb[b * 16 + i], S.d1[b * 64 + j], a);
                S.g[oW1 + q] += a;
            } else {
                const int j = q - 1024;
                float a = 0.f;
                for (int b = 0; b < nb; ++b) a += S.d1[b * 64 + j];
                S.g[oB1 + j] += a;
            }
        }
        __syncthreads();
    }
    if (tid == 0) S.loss *= invB;
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ X,
                                                   const int32_t* __restrict__ lab, int32_t B, float* __restrict__ grad,
                                                   float* __restrict__ loss) {
    extern __shared__ unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    for (int p = threadIdx.x; p < kNP; p += blockDim.x) S.th[p] = theta[p];
    __syncthreads();
    mlp_grad_block(S, X, lab, B);
    for (int p = threadIdx.x; p < kNP; p += blockDim.x) grad[p] = S.g[p];
    if (loss && threadIdx.x == 0) *loss = S.loss;
}

__device__ __forceinline__ void adam_update(float* th, const float* g, float* m, float* v, int p, float lr, float b1,
                                            float b2, float eps, float c1, float c2) {
    const float mm = b1 * m[p] + (1.f - b1) * g[p];
    const float vv = b2 * v[p] + (1.f - b2) * g[p] * g[p];
    m[p] = mm;
    v[p] = vv;
    th[p] = th[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int32_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) adam_update(th, g, m, v, p, lr, b1, b2, eps, c1, c2);
}

__global__ void __launch_bounds__(1024) k_mlp_train(float* __restrict__ theta, float* __restrict__ m,
                                                    float* __restrict__ v, const float* __restrict__ X,
                                                    const int32_t* __restrict__ lab, int32_t B, int32_t steps,
                                                    int32_t t0, float lr, float b1, float b2, float eps,
                                                    float* __restrict__ loss_hist) {
    extern __shared__ unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    for (int p = threadIdx.x; p < kNP; p += blockDim.x) S.th[p] = theta[p];
    __syncthreads();
    for (int st = 0; st < steps; ++st) {
        mlp_grad_block(S, X, lab, B);
        const int t = t0 + st + 1;
        const float c1 = 1.0f - powf(b1, (float)t);  // FP32: no FP64 in the training loop
        const float c2 = 1.0f - powf(b2, (float)t);
        for (int p = threadIdx.x; p < kNP; p += blockDim.x) adam_update(S.th, S.g, m, v, p, lr, b1, b2, eps, c1, c2);
        if (loss_hist && threadIdx.x == 0) loss_hist[st] = S.loss;
        __syncthreads();
    }
    for (int p = threadIdx.x; p < kNP; p += blockDim.x) theta[p] = S.th[p];
}

__global__ void k_mlp_scale(const float* __restrict__ f, const float* __restrict__ lo, const float* __restrict__ hi,
                            int32_t B, float* __restrict__ X) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < (int64_t)B * 16) X[q] = feat_scale((int)(q % 16), f[q], lo, hi);
}

__global__ void k_mlp_forward(const float* __restrict__ th, const float* __restrict__ X, int32_t B,
                              float* __restrict__ logits, int32_t* __restrict__ pred) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    float h1[64], h2[64], z[5];
    for (int j = 0; j < 64; ++j) {
        float a = th[oB1 + j];
        for (int i = 0; i < 16; ++i) a = fmaf(X[b * 16 + i], th[oW1 + i * 64 + j], a);
        h1[j] = a > 0.f ? a : 0.f;
    }
    for (int j = 0; j < 64; ++j) {
        float a = th[oB2 + j];
        for (int i = 0; i < 64; ++i) a = fmaf(h1[i], th[oW2 + i * 64 + j], a);
        h2[j] = a > 0.f ? a : 0.f;
    }
    int best = 0;
    for (int c = 0; c < 5; ++c) {
        float a = th[oB3 + c];
        for (int i = 0; i < 64; ++i) a = fmaf(h2[i], th[oW3 + i * 5 + c], a);
        z[c] = a;
        if (c > 0 && a > z[best]) best = c;
    }
    if (logits)
        for (int c = 0; c < 5; ++c) logits[b * 5 + c] = z[c];
    if (pred) pred[b] = best;
}

}  // namespace spmv

using namespace spmv;

extern "C" {

int spmv_features(const spmv_csr* csr, float* feat_dev, cudaStream_t stream) {
    if (!feat_dev) return set_error(SPMV_ERR_INVALID_ARG, "feat_dev is NULL");
    return launch_features(csr, feat_dev, nullptr, nullptr, nullptr, stream);
}

int spmv_model_create(const float* params_host, const float* lo_host, const float* hi_host, spmv_model** out) {
    if (!params_host || !lo_host || !hi_host || !out) return set_error(SPMV_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    spmv_model* md = new spmv_model();
    int st = dev_malloc((void**)&md->params, sizeof(float) * kNP);
    if (st == SPMV_OK) st = dev_malloc((void**)&md->lo, sizeof(float) * 16);
    if (st == SPMV_OK) st = dev_malloc((void**)&md->hi, sizeof(float) * 16);
    if (st == SPMV_OK) {
        cudaError_t e = cudaMemcpy(md->params, params_host, sizeof(float) * kNP, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(md->lo, lo_host, sizeof(float) * 16, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(md->hi, hi_host, sizeof(float) * 16, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_error(e, "spmv_model_create");
    }
    if (st == SPMV_OK) {
        spmv_params p{};
        md->max_bytes = resolve_cap(p);  // 90% of the memory free now
    }
    if (st != SPMV_OK) {
        dev_free(md->params);
        dev_free(md->lo);
        dev_free(md->hi);
        delete md;
        return st;
    }
    *out = md;
    return SPMV_OK;
}

int spmv_model_set_max_bytes(spmv_model* md, int64_t max_bytes) {
    if (!md || max_bytes <= 0) return set_error(SPMV_ERR_INVALID_ARG, "model is NULL or max_bytes <= 0");
    md->max_bytes = max_bytes;
    return SPMV_OK;
}

void spmv_model_free(spmv_model* md) {
    if (!md) return;
    dev_free(md->params);
    dev_free(md->lo);
    dev_free(md->hi);
    delete md;
}

int spmv_select_async(const spmv_csr* csr, const spmv_model* model, int32_t* fmt_dev, float* logits_dev,
                      cudaStream_t stream) {
    if (!model) return set_error(SPMV_ERR_NO_MODEL, "no selector model");
    if (!fmt_dev) return set_error(SPMV_ERR_INVALID_ARG, "fmt_dev is NULL");
    return launch_features(csr, nullptr, model, fmt_dev, logits_dev, stream);
}

int spmv_select(const spmv_csr* csr, const spmv_model* model, cudaStream_t stream, spmv_fmt* out) {
    if (!model) return set_error(SPMV_ERR_NO_MODEL, "no selector model");
    if (!out) return set_error(SPMV_ERR_INVALID_ARG, "out is NULL");
    static thread_local int32_t* d_fmt = nullptr;
    static thread_local int d_dev = -1;
    int dev = 0;
    SPMV_CUDA(cudaGetDevice(&dev));
    if (!d_fmt || d_dev != dev) {
        SPMV_TRY(dev_malloc((void**)&d_fmt, sizeof(int32_t)));
        d_dev = dev;
    }
    SPMV_TRY(launch_features(csr, nullptr, model, d_fmt, nullptr, stream));
    int32_t h = 0;
    SPMV_CUDA(cudaMemcpyAsync(&h, d_fmt, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    SPMV_CUDA(cudaStreamSynchronize(stream));
    *out = (spmv_fmt)h;
    return SPMV_OK;
}

int spmv_mlp_scale(const float* feat_dev, const float* lo_dev, const float* hi_dev, int32_t B, float* X_dev,
                   cudaStream_t stream) {
    if (!feat_dev || !lo_dev || !hi_dev || !X_dev || B < 0) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    if (B == 0) return SPMV_OK;
    k_mlp_scale<<<grid_for((int64_t)B * 16, 256), 256, 0, stream>>>(feat_dev, lo_dev, hi_dev, B, X_dev);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

static int train_smem_setup(const void* fn) {
    SPMV_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)));
    return SPMV_OK;
}

int spmv_mlp_loss_grad(const float* theta_dev, const float* X_dev, const int32_t* labels_dev, int32_t B,
                       float* grad_dev, float* loss_dev, cudaStream_t stream) {
    if (!theta_dev || !X_dev || !labels_dev || !grad_dev || B <= 0) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    SPMV_TRY(train_smem_setup((const void*)k_mlp_grad));
    k_mlp_grad<<<1, 1024, sizeof(TrainSmem), stream>>>(theta_dev, X_dev, labels_dev, B, grad_dev, loss_dev);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

int spmv_mlp_adam(float* theta_dev, const float* grad_dev, float* m_dev, float* v_dev, int32_t n, int32_t t, float lr,
                  float beta1, float beta2, float eps, cudaStream_t stream) {
    if (!theta_dev || !grad_dev || !m_dev || !v_dev || n <= 0 || t < 1) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)t));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)t));
    k_adam<<<grid_for(n, 256), 256, 0, stream>>>(theta_dev, grad_dev, m_dev, v_dev, n, lr, beta1, beta2, eps, c1, c2);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

int spmv_mlp_train(float* theta_dev, float* m_dev, float* v_dev, const float* X_dev, const int32_t* labels_dev,
                   int32_t B, int32_t steps, int32_t t0, float lr, float beta1, float beta2, float eps,
                   float* loss_hist_dev, cudaStream_t stream) {
    if (!theta_dev || !m_dev || !v_dev || !X_dev || !labels_dev || B <= 0 || steps < 0 || t0 < 0)
        return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    if (steps == 0) return SPMV_OK;
    SPMV_TRY(train_smem_setup((const void*)k_mlp_train));
    k_mlp_train<<<1, 1024, sizeof(TrainSmem), stream>>>(theta_dev, m_dev, v_dev, X_dev, labels_dev, B, steps, t0, lr,
                                                        beta1, beta2, eps, loss_hist_dev);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

int spmv_mlp_forward(const float* theta_dev, const float* X_dev, int32_t B, float* logits_dev, int32_t* pred_dev,
                     cudaStream_t stream) {
    if (!theta_dev || !X_dev || B < 0) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    if (B == 0) return SPMV_OK;
    k_mlp_forward<<<grid_for(B, 128), 128, 0, stream>>>(theta_dev, X_dev, B, logits_dev, pred_dev);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

}  // extern "C"
