// Matrix features (Sec. V-B "Features", Table IV), their scaling (Sec. V-B
// "Feature Scaling") and the selector network (Sec. V-A/V-B: features in,
// representation label out; here a 16-64-64-5 multilayer perceptron, one of
// the alternatives of Sec. V-D), with its training kernels.
//
// Feature definitions (rows sampled when M > 8192):
//   R = all rows, or rows floor(k*M/8192) for k < 8192; len_i = ptr[i+1]-ptr[i]
//   0 n_rows  1 n_cols  2 nnz/(M*N)  3 min len  4 max len  5 nnz/M
//   6 std of len over R  7 std/mean  8 log2(max(nnz,1))  9 mean/max
//  10 HYB tail fraction with K from R (lengths capped at 512)
//  11 mean |col-row| and 12 max |col-row| over the first 16 entries of each sampled row
//  13 fraction of empty rows  14 fraction of rows with len >= 32
//  15 SELL-32 fill over R sorted, lengths capped at 512
//
// The features kernel is one cluster of 8 CTAs x 1024 threads: each CTA
// reduces its share of the sampled rows, then CTA 0 combines the eight
// partial results through distributed shared memory (no global scratch, no
// atomics across CTAs) and, for selection, runs the network.
#include <cooperative_groups.h>
#include <cuda_pipeline.h>

#include "internal.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

struct spmv_model {
    float* params = nullptr;  // SPMV_MLP_PARAMS
    float* lo = nullptr;      // 16
    float* hi = nullptr;      // 16
};

namespace spmv {

constexpr int kFeatCtas = 8;
constexpr int kFeatThreads = 1024;
constexpr int kSample = 8192;  // = kFeatCtas * kFeatThreads: one sampled row per thread
constexpr int kLenCap = 512;
constexpr int kSpread = 16;

// parameter offsets inside the flat vector
constexpr int oW1 = 0, oB1 = 1024, oW2 = 1088, oB2 = 5184, oW3 = 5248, oB3 = 5568, kNP = 5573;

struct FeatStats {  // one CTA's partial statistics of the sampled rows
    unsigned long long sum_len, sum_sq, spread_sum, spread_cnt;
    int min_len, max_len, band;
    unsigned empty, longc;
};

// Transform and min-max scaling of one feature.  FP32 on purpose: this GPU's
// FP64 pipe makes double log2/division/sqrt several microseconds slower, and
// the features are float32 values to begin with.
__device__ __forceinline__ float feat_transform(int j, float f) {
    if (j == 0 || j == 1 || j == 3 || j == 4 || j == 5 || j == 6 || j == 11 || j == 12) return log2f(1.0f + f);
    if (j == 2) return -log2f(fmaxf(f, 0x1.0p-60f));
    return f;
}

__device__ __forceinline__ float feat_scale(int j, float f, const float* lo, const float* hi) {
    const float t = feat_transform(j, f);
    const float span = hi[j] - lo[j];
    if (!(span > 0.0f)) return 0.0f;
    const float x = (t - lo[j]) / span;
    return x < 0.0f ? 0.0f : (x > 1.0f ? 1.0f : x);
}

// Barrier of the first two warps only (named barrier 1), for the tail of the
// features kernel that runs in warps 0 and 1 after the others have left.
__device__ __forceinline__ void tail_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// 16 -> 64 -> 64 -> 5 forward for one sample in threads 0..63 (warps 0 and 1);
// th in shared memory.  Thread j computes hidden unit j of each layer as one
// dot product (consecutive j: conflict-free weight reads, broadcast inputs).
__device__ void mlp_forward_64(const float* th, const float* xs, float* h1, float* h2, float* z) {
    const int j = threadIdx.x;
    float a = th[oB1 + j];
#pragma unroll
    for (int i = 0; i < 16; ++i) a = fmaf(xs[i], th[oW1 + i * 64 + j], a);
    h1[j] = a > 0.f ? a : 0.f;
    tail_sync();
    a = th[oB2 + j];
#pragma unroll 16
    for (int i = 0; i < 64; ++i) a = fmaf(h1[i], th[oW2 + i * 64 + j], a);
    h2[j] = a > 0.f ? a : 0.f;
    tail_sync();
    if (j < 5) {
        a = th[oB3 + j];
#pragma unroll 16
        for (int i = 0; i < 64; ++i) a = fmaf(h2[i], th[oW3 + i * 5 + j], a);
        z[j] = a;
    }
    tail_sync();
}

__global__ void __cluster_dims__(kFeatCtas, 1, 1) __launch_bounds__(kFeatThreads)
    k_features(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, int32_t m, int32_t n,
               float* __restrict__ feat_out, const float* __restrict__ model_params, const float* __restrict__ lo,
               const float* __restrict__ hi, int32_t* __restrict__ fmt_out, float* __restrict__ logits_out) {
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    __shared__ unsigned hist[kLenCap + 1];                // this CTA's length histogram
    __shared__ FeatStats parts[kFeatCtas];                // in CTA 0: every CTA's statistics
    __shared__ unsigned hists[kFeatCtas * (kLenCap + 1)]; // in CTA 0: every CTA's histogram
    __shared__ unsigned long long red_u[32][4];
    __shared__ int red_i[32][3];
    __shared__ unsigned red_c[32][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // CTA 0 starts copying what its tail needs into shared memory now
    // (asynchronous copies, waited for just before the tail): nnz = ptr[m]
    // and, for a selection, the network and the scaling table.
    __shared__ __align__(16) float wsm[kNP + 3 + 32];
    __shared__ int32_t nnz_sm;
    if (rank == 0) {
        if (tid == 0) __pipeline_memcpy_async(&nnz_sm, ptr + m, 4);
        if (model_params) {
            for (int c = tid; c < kNP / 4; c += kFeatThreads) __pipeline_memcpy_async(wsm + 4 * c, model_params + 4 * c, 16);
            if (tid < kNP % 4) __pipeline_memcpy_async(wsm + (kNP / 4) * 4 + tid, model_params + (kNP / 4) * 4 + tid, 4);
            if (tid < 4) __pipeline_memcpy_async(wsm + kNP + 3 + 4 * tid, lo + 4 * tid, 16);
            else if (tid < 8) __pipeline_memcpy_async(wsm + kNP + 3 + 16 + 4 * (tid - 4), hi + 4 * (tid - 4), 16);
        }
        __pipeline_commit();
    }
    for (int b = tid; b <= kLenCap; b += kFeatThreads) hist[b] = 0;
    __syncthreads();

    // ---- phase 1: every CTA reduces its share of the sampled rows, one per
    // thread (8 CTAs x 1024 threads, 8192 samples).  Row of sample k: k*M/S,
    // with S = 8192 = 2^13 whenever M > S (a shift), else k.
    const int64_t S = m < kSample ? m : kSample;
    unsigned long long sl = 0, sq = 0, ssum = 0, scnt = 0;
    int mn = 0x7fffffff, mx = 0, band = 0;
    unsigned emp = 0, lng = 0;
    {
        constexpr int kRows = kSample / (kFeatCtas * kFeatThreads);  // sampled rows per thread
        static_assert(kSample == kFeatCtas * kFeatThreads * kRows && kSample == 1 << 13, "sample layout");
        int64_t kk[kRows], ii[kRows];
        int32_t p0[kRows], p1[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            kk[r] = (int64_t)rank * kFeatThreads + tid + (int64_t)r * kFeatCtas * kFeatThreads;
            ii[r] = m > kSample ? ((kk[r] * (int64_t)m) >> 13) : kk[r];
            const bool on = kk[r] < S;
            p0[r] = on ? ptr[ii[r]] : 0;
            p1[r] = on ? ptr[ii[r] + 1] : 0;
        }
        int32_t c[kRows][kSpread];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int32_t len = p1[r] - p0[r];
            const int ne = len < kSpread ? len : kSpread;
#pragma unroll
            for (int q = 0; q < kSpread; ++q) c[r][q] = q < ne ? __ldg(idx + p0[r] + q) : (int32_t)ii[r];
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const bool on = kk[r] < S;
            const int32_t len = p1[r] - p0[r];
            if (on) {
                sl += (unsigned long long)len;
                sq += (unsigned long long)len * (unsigned long long)len;
                mn = min(mn, len);
                mx = max(mx, len);
                emp += len == 0;
                lng += len >= 32;
                scnt += (unsigned long long)(len < kSpread ? len : kSpread);
#pragma unroll
                for (int q = 0; q < kSpread; ++q) {
                    const int64_t d = (int64_t)c[r][q] - ii[r];
                    const int ad = (int)(d < 0 ? -d : d);
                    ssum += (unsigned long long)ad;
                    band = max(band, ad);
                }
            }
            // one shared atomic per distinct bin in the warp
            const unsigned act = __ballot_sync(dev::kFull, on);
            if (on) {
                const int bin = len < kLenCap ? len : kLenCap;
                const unsigned peers = __match_any_sync(act, bin);
                if (lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sl += __shfl_xor_sync(dev::kFull, sl, o);
        sq += __shfl_xor_sync(dev::kFull, sq, o);
        ssum += __shfl_xor_sync(dev::kFull, ssum, o);
        scnt += __shfl_xor_sync(dev::kFull, scnt, o);
        mn = min(mn, __shfl_xor_sync(dev::kFull, mn, o));
        mx = max(mx, __shfl_xor_sync(dev::kFull, mx, o));
        band = max(band, __shfl_xor_sync(dev::kFull, band, o));
        emp += __shfl_xor_sync(dev::kFull, emp, o);
        lng += __shfl_xor_sync(dev::kFull, lng, o);
    }
    if (lane == 0) {
        red_u[warp][0] = sl; red_u[warp][1] = sq; red_u[warp][2] = ssum; red_u[warp][3] = scnt;
        red_i[warp][0] = mn; red_i[warp][1] = mx; red_i[warp][2] = band;
        red_c[warp][0] = emp; red_c[warp][1] = lng;
    }
    __syncthreads();
    // push this CTA's partial into CTA 0's shared memory; one cluster barrier publishes them.
    // Warp 0 combines the 32 warp partials with shuffles.
    if (warp == 0) {
        unsigned long long a0 = red_u[lane][0], a1 = red_u[lane][1], a2 = red_u[lane][2], a3 = red_u[lane][3];
        int i0 = red_i[lane][0], i1 = red_i[lane][1], i2 = red_i[lane][2];
        unsigned c0 = red_c[lane][0], c1 = red_c[lane][1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(dev::kFull, a0, o);
            a1 += __shfl_xor_sync(dev::kFull, a1, o);
            a2 += __shfl_xor_sync(dev::kFull, a2, o);
            a3 += __shfl_xor_sync(dev::kFull, a3, o);
            i0 = min(i0, __shfl_xor_sync(dev::kFull, i0, o));
            i1 = max(i1, __shfl_xor_sync(dev::kFull, i1, o));
            i2 = max(i2, __shfl_xor_sync(dev::kFull, i2, o));
            c0 += __shfl_xor_sync(dev::kFull, c0, o);
            c1 += __shfl_xor_sync(dev::kFull, c1, o);
        }
        if (lane == 0) {
            FeatStats p;
            p.sum_len = a0; p.sum_sq = a1; p.spread_sum = a2; p.spread_cnt = a3;
            p.min_len = i0; p.max_len = i1; p.band = i2; p.empty = c0; p.longc = c1;
            *cluster.map_shared_rank(&parts[rank], 0) = p;
        }
    }
    unsigned* h0 = cluster.map_shared_rank(hists, 0);
    for (int b = tid; b <= kLenCap; b += kFeatThreads) h0[rank * (kLenCap + 1) + b] = hist[b];
    cluster.sync();
    if (rank != 0) return;  // CTA 0 holds everything now

    // ---- phase 2 (CTA 0): combine, features, optional selection.  The
    // histogram ranks are summed by 513 threads; the rest runs in warps 0
    // and 1 (the scans in warp 0 with shuffles only, lane l owning bins
    // 17l .. 17l + 16; the network in both warps).
    __shared__ unsigned hsum[kLenCap + 1];
    __shared__ FeatStats tot;
    __shared__ float fs[16], xs[16], h1[64], h2[64], z[5];
    if (tid <= kLenCap) {
        unsigned v = 0;
#pragma unroll
        for (int r = 0; r < kFeatCtas; ++r) v += hists[r * (kLenCap + 1) + tid];
        hsum[tid] = v;
    }
    if (warp == 0) {  // combine the eight CTA partials (lanes 0..7) with shuffles
        const int r = lane < kFeatCtas ? lane : 0;
        const bool on = lane < kFeatCtas;
        unsigned long long a0 = on ? parts[r].sum_len : 0, a1 = on ? parts[r].sum_sq : 0;
        unsigned long long a2 = on ? parts[r].spread_sum : 0, a3 = on ? parts[r].spread_cnt : 0;
        int i0 = on ? parts[r].min_len : 0x7fffffff, i1 = on ? parts[r].max_len : 0, i2 = on ? parts[r].band : 0;
        unsigned c0 = on ? parts[r].empty : 0, c1 = on ? parts[r].longc : 0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(dev::kFull, a0, o);
            a1 += __shfl_xor_sync(dev::kFull, a1, o);
            a2 += __shfl_xor_sync(dev::kFull, a2, o);
            a3 += __shfl_xor_sync(dev::kFull, a3, o);
            i0 = min(i0, __shfl_xor_sync(dev::kFull, i0, o));
            i1 = max(i1, __shfl_xor_sync(dev::kFull, i1, o));
            i2 = max(i2, __shfl_xor_sync(dev::kFull, i2, o));
            c0 += __shfl_xor_sync(dev::kFull, c0, o);
            c1 += __shfl_xor_sync(dev::kFull, c1, o);
        }
        if (lane == 0) {
            tot.sum_len = a0; tot.sum_sq = a1; tot.spread_sum = a2; tot.spread_cnt = a3;
            tot.min_len = i0; tot.max_len = i1; tot.band = i2; tot.empty = c0; tot.longc = c1;
        }
    }
    __pipeline_wait_prior(0);  // this thread's copies of nnz and the network have landed
    __syncthreads();
    if (tid >= 64) return;
    const unsigned cnt = (unsigned)S;
    unsigned long long upto_k = 0, widths = 0, capped_sum = 0;
    if (warp == 0) {
        // c_b = #{len >= b}: suffix sums over the bins (in-lane, then over the lanes)
        constexpr int PB = 17;  // bins per lane: 32 * 17 = 544 >= 513
        unsigned c[PB];
        unsigned run = 0;
#pragma unroll
        for (int j = PB - 1; j >= 0; --j) {
            const int bb = lane * PB + j;
            run += bb <= kLenCap ? hsum[bb] : 0u;
            c[j] = run;  // in-lane suffix
        }
        unsigned later = run;  // this lane's total, then the totals of later lanes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_down_sync(dev::kFull, later, d);
            if (lane + d < 32) later += u;
        }
        later -= run;
        const unsigned need = (cnt + 2) / 3;
        unsigned long long k_ok = 0, wpart = 0, cpart = 0;
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            const int bb = lane * PB + j;
            c[j] += later;
            if (bb >= 1 && bb <= kLenCap) {
                k_ok += c[j] >= need;
                wpart += (c[j] + 31) / 32;
                cpart += c[j];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            k_ok += __shfl_xor_sync(dev::kFull, k_ok, o);
            wpart += __shfl_xor_sync(dev::kFull, wpart, o);
            cpart += __shfl_xor_sync(dev::kFull, cpart, o);
        }
        const int K = (int)k_ok;  // c_b is non-increasing, so the bins >= need are 1..K
        unsigned long long up = 0;
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            const int bb = lane * PB + j;
            if (bb >= 1 && bb <= K) up += c[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) up += __shfl_xor_sync(dev::kFull, up, o);
        upto_k = up;  // sum min(len, K)
        widths = wpart;
        capped_sum = cpart;
    }
    if (tid < 16) {  // one lane per feature, FP32 (exact integer parts kept in 64 bits)
        // Every lane evaluates the same straight-line code (no divergent
        // per-feature paths) and keeps its own feature.
        const int j = tid;
        const float fc = (float)cnt;
        const float L = (float)tot.sum_len;
        const float mean = L / fc;
        const float nnz = (float)nnz_sm;
        // std = sqrt(cnt * sum_sq - L^2) / cnt, the difference in exact 128-bit integer arithmetic
        const unsigned long long a_lo = (unsigned long long)cnt * tot.sum_sq;
        const unsigned long long a_hi = __umul64hi((unsigned long long)cnt, tot.sum_sq);
        const unsigned long long b_lo = tot.sum_len * tot.sum_len;
        const unsigned long long b_hi = __umul64hi(tot.sum_len, tot.sum_len);
        const unsigned long long d_lo = a_lo - b_lo;
        const unsigned long long d_hi = a_hi - b_hi - (a_lo < b_lo ? 1ull : 0ull);
        const float sd = sqrtf((float)d_hi * 18446744073709551616.0f + (float)d_lo) / fc;
        // the quotient and the log each lane needs, selected before the one division and log2
        float num = 0.0f, den = 1.0f;
        switch (j) {
            case 2: num = nnz; den = (float)m * (float)n; break;
            case 5: num = nnz; den = (float)m; break;
            case 7: num = tot.sum_len > 0 ? sd : 0.0f; den = tot.sum_len > 0 ? mean : 1.0f; break;
            case 9: num = tot.max_len > 0 ? mean : 0.0f; den = tot.max_len > 0 ? (float)tot.max_len : 1.0f; break;
            case 10: num = tot.sum_len > 0 ? (float)(tot.sum_len - upto_k) : 0.0f; den = tot.sum_len > 0 ? L : 1.0f; break;
            case 11: num = tot.spread_cnt > 0 ? (float)tot.spread_sum : 0.0f; den = tot.spread_cnt > 0 ? (float)tot.spread_cnt : 1.0f; break;
            case 13: num = (float)tot.empty; den = fc; break;
            case 14: num = (float)tot.longc; den = fc; break;
            case 15: num = widths > 0 ? (float)capped_sum : 1.0f; den = widths > 0 ? 32.0f * (float)widths : 1.0f; break;
            default: break;
        }
        const float q = num / den;
        const float lg = log2f(nnz > 1.0f ? nnz : 1.0f);
        float f = q;
        if (j == 0) f = (float)m;
        if (j == 1) f = (float)n;
        if (j == 3) f = (float)tot.min_len;
        if (j == 4) f = (float)tot.max_len;
        if (j == 6) f = sd;
        if (j == 8) f = lg;
        if (j == 12) f = (float)tot.band;
        fs[j] = f;
    }
    tail_sync();
    if (feat_out && tid < 16) feat_out[tid] = fs[tid];
    if (model_params) {
        if (tid < 16) xs[tid] = feat_scale(tid, fs[tid], wsm + kNP + 3, wsm + kNP + 3 + 16);
        tail_sync();
        mlp_forward_64(wsm, xs, h1, h2, z);
        if (tid == 0) {
            int best = 0;
            for (int c = 1; c < 5; ++c)
                if (z[c] > z[best]) best = c;
            if (fmt_out) fmt_out[0] = best;
        }
        if (logits_out && tid < 5) logits_out[tid] = z[tid];
    }
}

static int launch_features(const spmv_csr* c, float* feat, const spmv_model* model, int32_t* fmt, float* logits,
                           cudaStream_t s) {
    if (!c) return set_error(SPMV_ERR_INVALID_ARG, "csr is NULL");
    if (c->m <= 0 || c->n <= 0 || !c->ptr || (c->nnz > 0 && !c->idx))
        return set_error(SPMV_ERR_INVALID_ARG, "malformed csr argument");
    k_features<<<kFeatCtas, kFeatThreads, 0, s>>>(c->ptr, c->idx, c->m, c->n, feat, model ? model->params : nullptr,
                                                 model ? model->lo : nullptr, model ? model->hi : nullptr, fmt, logits);
    SPMV_CUDA(cudaGetLastError());
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
