// Device-side work units of the five formats.  Each function processes one
// unit of one matrix and is called both by that format's own kernel and by the
// batched persistent kernel, so the two paths run the same arithmetic.
//
// Loads: matrix data (values, column indices) is read once per product and
// goes through the streaming path (ld.global.cs, evict-first); x is gathered
// through the read-only path (ld.global.nc) so it stays resident in L2.
#pragma once

#include <cstdint>
#include <cuda/atomic>
#include <cuda_runtime.h>

namespace spmv {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start before the kernel ahead of it in the stream has
// finished; pdl_wait() blocks until that kernel has completed and its memory
// is visible (a no-op for an ordinary launch).  pdl_trigger() lets the next
// such kernel start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double ldx(const double* x, int32_t c) { return __ldg(x + c); }

// Row of nonzero k: the largest i with ptr[i] <= k (empty rows are skipped).
__device__ __forceinline__ int32_t row_of_nnz(const int32_t* __restrict__ ptr, int32_t m, int64_t k) {
    int32_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo + 1) / 2;
        if (ptr[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum over a 256-thread block; the result is valid in thread 0.  red: 8 doubles.
__device__ __forceinline__ double block_sum256(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) s += red[i];
    }
    return s;
}

// ------------------------------------------------------------------- CSR
//
// On this GPU the FP64 pipe issues about two lanes per clock per SM, so every
// FP64 instruction must carry a full warp of useful work: one DFMA per
// nonzero, lanes kept busy, cross-lane FP64 reductions only where amortised.
// Random gathers of x cost one L1 wavefront per lane, so every other load is
// coalesced.
//
// The CSR arrays are used as they are; the work is cut by nonzeros, not by
// rows: tile u is nonzeros [u*W, (u+1)*W) (W = 32*kCsrCT), one warp each, so
// every warp carries the same load whatever the row lengths.  A row gets
// lanes in proportion to its length: a lane walks many short rows, a long row
// spans many lanes or tiles.  The warp
//  1. stages the tile's values and column indices in its shared slice with
//     coalesced loads;
//  2. reads the pointers of the rows that start in the tile (rows
//     tile_row[u] .. tile_row[u+1]-1), writes y = 0 for the empty ones, and
//     for each nonempty one sets a bit in a per-lane flag word (bit r of
//     lane l: nonzero l*kCsrCT + r begins a row) and appends its row number
//     to the tile's segment list (ballots keep the list in row order);
//  3. lane l walks its kCsrCT nonzeros with one gather and one DFMA each,
//     writing every row that begins and ends in its chunk; a segmented
//     suffix sum over the lanes (shuffles) completes the rows spanning lanes;
//  4. a tile owns the rows that begin in it.  When its last row runs past
//     the tile end by at most W nonzeros, the warp reads that overflow itself
//     (coalesced, one warp reduction) and the next tile skips the row's head
//     without gathering it.  A longer row is finished by the last of its
//     tiles to arrive: each stores its part in a per-tile slot and takes a
//     ticket, and the last ticket holder adds the slots in tile order (no
//     waiting, deterministic order).
constexpr int kCsrCT = 11;          // nonzeros per lane (odd: conflict-free shared accesses)
constexpr int kCsrW = 32 * kCsrCT;  // nonzeros per tile

struct CsrArgs {
    const int32_t* tile_row;  // ntiles + 1: first row with ptr >= u*W; tile_row[ntiles] = rows
    const int32_t* ptr;
    const int32_t* idx;
    const double* val;
    const int32_t* row_map;   // ADD mode: y[row_map[r]] += sum; else y[r] = sum
    double* slot_head;        // per tile: its part of a row begun in an earlier tile
    double* slot_tail;        // per tile: its open last segment
    unsigned* cnt;            // per start tile: tickets of the row's tiles (reset after use)
    int32_t rows;
    int32_t nnz;
    int32_t ntiles;
    const double* x;
    double* y;
};

struct CsrWarpSmem {
    double sv[kCsrW];
    int32_t si[kCsrW];
    int32_t rid[kCsrW + 1];  // row of each segment of the tile, in order
    uint32_t fl[32];
};
constexpr int kCsrWarps = 8;  // warps (tiles in flight) per 256-thread block
constexpr size_t kCsrSmemBytes = sizeof(CsrWarpSmem) * kCsrWarps;

template <bool ADD>
__device__ __forceinline__ void csr_put(const CsrArgs& a, int32_t r, double s) {
    if (ADD) {
        const int32_t rr = a.row_map[r];
        a.y[rr] += s;
    } else {
        a.y[r] = s;
    }
}

// Rows of similar length: row r by V lanes (lane = this thread's place among
// them).  Each lane keeps a strided share of the row's entries, the row's
// lanes reading consecutive addresses together, and a shuffle tree over the
// V lanes closes the row.  Every thread of the warp must call this (rows past
// the end contribute nothing).
template <int V>
__device__ __forceinline__ void csr_lanes_row(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                              const double* __restrict__ val, const double* __restrict__ x,
                                              double* __restrict__ y, int32_t m, int64_t r, int lane) {
    double s = 0.0;
    if (r < m) {
        const int32_t p1 = ptr[r + 1];
        for (int32_t k = ptr[r] + lane; k < p1; k += V) s = fma(__ldcs(val + k), ldx(x, __ldcs(idx + k)), s);
    }
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o, V);
    if (r < m && lane == 0) y[r] = s;
}

// Tile t's part v of row r (tail: r begins in t; else r began earlier).
template <bool ADD>
__device__ __forceinline__ void csr_join(const CsrArgs& a, int32_t r, int32_t t, bool tail, double v) {
    const uint32_t t0 = (uint32_t)a.ptr[r] / (uint32_t)kCsrW;
    const uint32_t t1 = ((uint32_t)a.ptr[r + 1] - 1u) / (uint32_t)kCsrW;
    if (tail) a.slot_tail[t] = v;
    else a.slot_head[t] = v;
    // release our slot, acquire the others' (the last ticket sees every slot)
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> ticket(a.cnt[t0]);
    const unsigned prev = ticket.fetch_add(1u, cuda::memory_order_acq_rel);
    if (prev == t1 - t0) {
        double acc = __ldcg(a.slot_tail + t0);
#pragma unroll 8
        for (uint32_t u = t0 + 1; u <= t1; ++u) acc += __ldcg(a.slot_head + u);
        ticket.store(0u, cuda::memory_order_relaxed);
        csr_put<ADD>(a, r, acc);
    }
}

template <bool ADD>
__device__ __forceinline__ void csr_tile(const CsrArgs& a, int32_t t, CsrWarpSmem& S, int lane) {
    const int64_t base = (int64_t)t * kCsrW;
    const int32_t n = (int32_t)min((int64_t)kCsrW, (int64_t)a.nnz - base);  // >= 1
    const int32_t r0 = a.tile_row[t], r1 = a.tile_row[t + 1];
    // 1. stage values and column indices (coalesced)
    const double* __restrict__ vb = a.val + base;
    const int32_t* __restrict__ ib = a.idx + base;
    if (n == kCsrW) {
#pragma unroll
        for (int q = 0; q < kCsrCT; ++q) {
            S.sv[q * 32 + lane] = __ldcs(vb + q * 32 + lane);
            S.si[q * 32 + lane] = __ldcs(ib + q * 32 + lane);
        }
    } else {
        for (int j = lane; j < n; j += 32) {
            S.sv[j] = __ldcs(vb + j);
            S.si[j] = __ldcs(ib + j);
        }
    }
    S.fl[lane] = lane == 0 ? 1u : 0u;  // the tile's first nonzero always opens a segment
    __syncwarp();
    // 2. the rows starting in the tile
    const int32_t p_r0 = a.ptr[r0];
    const int32_t p_r1 = a.ptr[r1];      // end of the tile's last row
    const bool cont = p_r0 > base;       // nonzero `base` lies in row r0 - 1, begun earlier
    // that row is finished by the tile it began in when it overflows that tile by <= W
    bool skip_head = false;
    if (cont) {
        const int64_t ts = a.ptr[r0 - 1] / kCsrW;
        skip_head = (int64_t)p_r0 - (ts + 1) * kCsrW <= kCsrW;
    }
    const int32_t head_end = (int32_t)((int64_t)p_r0 - base);  // tile position after that row
    if (cont && lane == 0) S.rid[0] = r0 - 1;
    int32_t nseg = cont ? 1 : 0;
    for (int32_t rb = r0; rb < r1; rb += 32) {
        const int32_t r = rb + lane;
        int32_t p = 0;
        bool nonempty = false;
        if (r < r1) {
            p = a.ptr[r];
            nonempty = a.ptr[r + 1] > p;
            if (!ADD && !nonempty) a.y[r] = 0.0;
        }
        const unsigned mask = __ballot_sync(kFull, nonempty);
        if (nonempty) {
            const int32_t pos = (int32_t)(p - base);
            S.rid[nseg + __popc(mask & ((1u << lane) - 1u))] = r;
            atomicOr(&S.fl[pos / kCsrCT], 1u << (pos % kCsrCT));
        }
        nseg += __popc(mask);
    }
    __syncwarp();
    // 3. the walk
    const uint32_t f = S.fl[lane];
    const int nf = __popc(f);
    int yo = nf;  // inclusive count of flags up to this lane
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(kFull, yo, d);
        if (lane >= d) yo += v;
    }
    const int total = __shfl_sync(kFull, yo, 31);  // segments in the tile
    yo -= nf;
    const int c0 = lane * kCsrCT;
    double cur = 0.0, head = 0.0;
    double first = 0.0;  // lane 0: segment 0 when it continues a row and closes inside the lane
    bool first_join = false;
    int j = 0;  // segments of this lane seen so far
#pragma unroll
    for (int r = 0; r < kCsrCT; ++r) {
        const int k = c0 + r;
        const bool valid = k < n && !(skip_head && k < head_end);  // past the end, or another tile's row
        const double v = valid ? S.sv[k] : 0.0;
        const double xv = valid ? ldx(a.x, S.si[k]) : 0.0;
        if ((f >> r) & 1u) {
            if (j == 0) {
                head = cur;
            } else {  // segment yo + j - 1 ends here, complete within the tile
                const int g = yo + j - 1;
                if (g == 0 && cont) {  // joined after the walk, keeping the loop lean
                    first = cur;
                    first_join = true;
                } else {
                    csr_put<ADD>(a, S.rid[g], cur);
                }
            }
            ++j;
            cur = 0.0;
        }
        cur = fma(v, xv, cur);  // one DFMA per nonzero
    }
    if (nf == 0) head = cur;
    // T_l = head_l + (lane l holds no flag ? T_{l+1} : 0)
    double T = head;
    int stop = nf > 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double Tn = __shfl_down_sync(kFull, T, d);
        const int sn = __shfl_down_sync(kFull, stop, d);
        if (!stop && lane + d < 32) {
            T += Tn;
            stop = sn;
        }
    }
    double next = __shfl_down_sync(kFull, T, 1);
    if (lane == 31) next = 0.0;
    // 4. the lane's last segment, and the rows crossing tiles
    const bool crosses = (int64_t)p_r1 > base + kCsrW && !(total == 1 && cont);  // a row begun here runs on
    const bool own_overflow = crosses && (int64_t)p_r1 - (base + kCsrW) <= kCsrW;  // warp-uniform
    double ov = 0.0;
    if (own_overflow) {
        for (int64_t k = base + kCsrW + lane; k < p_r1; k += 32) ov = fma(__ldcs(a.val + k), ldx(a.x, __ldcs(a.idx + k)), ov);
        ov = warp_sum(ov);
    }
    if (first_join && !skip_head) csr_join<ADD>(a, r0 - 1, t, false, first);
    if (nf > 0) {
        const int g = yo + nf - 1;
        const int32_t row = S.rid[g];
        const double tot = cur + next;
        if (g == 0 && cont) {  // continues a row begun in an earlier tile
            if (!skip_head) csr_join<ADD>(a, row, t, false, tot);
        } else if (g == total - 1 && crosses) {  // begins here, continues into later tiles
            if (own_overflow) csr_put<ADD>(a, row, tot + ov);
            else csr_join<ADD>(a, row, t, true, tot);
        } else {
            csr_put<ADD>(a, row, tot);
        }
    }
    __syncwarp();  // the shared slice is reused by the warp's next tile
}

// y = 0 for the rows of a matrix without nonzeros (no tiles).
__device__ __forceinline__ void csr_zero(const CsrArgs& a, int64_t i) {
    if (i < a.rows) a.y[i] = 0.0;
}

// ------------------------------------------------------------------- ELL
//
// Column-major ELL (slot s of row i at s*ld + i, ld even): thread t handles
// rows 2t and 2t+1 with one 16-byte value load and one 8-byte index load per
// slot, bounded by row_len so padding never reaches a product.  Rows longer
// than long_len are left to ell_long_row (y not written here).
struct EllArgs {
    const int32_t* row_len;
    const int32_t* col;
    const double* val;
    int64_t ld;
    int32_t m;
    int32_t long_len;
    const double* x;
    double* y;
};

__device__ __forceinline__ void ell_rows2(const EllArgs& a, int32_t i0) {
    if (i0 >= a.m) return;
    const int2 L = *reinterpret_cast<const int2*>(a.row_len + i0);
    const int32_t l0 = L.x > a.long_len ? 0 : L.x;
    const int32_t l1 = L.y > a.long_len ? 0 : L.y;
    const int32_t lm = l0 > l1 ? l0 : l1;
    double s0 = 0.0, s1 = 0.0;
    const double2* v2 = reinterpret_cast<const double2*>(a.val + i0);
    const int2* c2 = reinterpret_cast<const int2*>(a.col + i0);
    const int64_t st = a.ld >> 1;
#pragma unroll 4
    for (int32_t s = 0; s < lm; ++s) {
        const double2 v = __ldcs(v2 + s * st);
        const int2 c = __ldcs(c2 + s * st);
        if (s < l0) s0 = fma(v.x, ldx(a.x, c.x), s0);
        if (s < l1) s1 = fma(v.y, ldx(a.x, c.y), s1);
    }
    if (L.x <= a.long_len) a.y[i0] = s0;
    if (i0 + 1 < a.m && L.y <= a.long_len) a.y[i0 + 1] = s1;
}

// One long ELL row by a 256-thread block (slots strided by ld).
__device__ __forceinline__ void ell_long_row(const EllArgs& a, int32_t i, double* red) {
    const int32_t len = a.row_len[i];
    double s0 = 0.0, s1 = 0.0;
    int32_t s = threadIdx.x;
    for (; s + 256 < len; s += 512) {
        const int64_t o0 = (int64_t)s * a.ld + i, o1 = (int64_t)(s + 256) * a.ld + i;
        s0 = fma(__ldcs(a.val + o0), ldx(a.x, __ldcs(a.col + o0)), s0);
        s1 = fma(__ldcs(a.val + o1), ldx(a.x, __ldcs(a.col + o1)), s1);
    }
    for (; s < len; s += 256) {
        const int64_t o = (int64_t)s * a.ld + i;
        s0 = fma(__ldcs(a.val + o), ldx(a.x, __ldcs(a.col + o)), s0);
    }
    const double t = block_sum256(s0 + s1, red);
    if (threadIdx.x == 0) a.y[i] = t;
    __syncthreads();
}

// ----------------------------------------------------------- SELL-C-sigma
//
// A warp processes one unit {slice, chunk}: lane l holds the R = C/32 sorted
// positions s*C + l*R .. + R-1, reading R values and R indices per slot with
// vector loads (R = 2: 16 + 8 bytes, R = 4: 2 x 16 + 16 bytes).  Wide slices
// are split into chunks of `unit_width` slots whose partial sums are added in
// chunk order by the last chunk to finish.  The row sums go out by MODE:
//   kSellPlain  y[perm[pos]] = sum    (one SELL matrix)
//   kSellFirst  ys[pos] = sum          (column panels sharing one row order:
//   kSellMid    ys[pos] += sum          the partial sums stay in sorted order,
//                                       coalesced; a last pass puts them back
//                                       in row order)
struct SellArgs {
    const int2* units;
    const int64_t* slice_ptr;
    const int32_t* len;   // per sorted position, padded to a multiple of C
    const int32_t* perm;  // sorted position -> row
    const int32_t* col;
    const double* val;
    double* partial;
    unsigned* counters;
    int32_t m;
    int32_t unit_width;
    const double* x;
    double* y;
    double* ys;           // panels: partial sums per sorted position
};

enum SellOut : int { kSellPlain = 0, kSellFirst = 1, kSellMid = 2, kSellIdent = 3 };

// perm and the sorted-order partial sums are streamed (evict-first loads,
// streaming stores), so that they do not push x out of L2; the scattered y
// stores keep the default policy, so that neighbouring rows' writes can meet
// in L2 before a sector goes to memory.
template <int MODE>
__device__ __forceinline__ void sell_put(const SellArgs& a, int64_t pos, double v) {
    if constexpr (MODE == kSellPlain) a.y[__ldcs(a.perm + pos)] = v;
    else if constexpr (MODE == kSellIdent) __stcs(a.y + pos, v);  // the sort left every row in place
    else if constexpr (MODE == kSellFirst) __stcs(a.ys + pos, v);
    else __stcs(a.ys + pos, __ldcs(a.ys + pos) + v);
}

template <int R, int MODE = kSellPlain>
__device__ __forceinline__ void sell_unit(const SellArgs& a, int32_t u, int lane) {
    constexpr int C = 32 * R;
    const int2 U = a.units[u];
    const int64_t base = a.slice_ptr[U.x];
    const int32_t w = (int32_t)((a.slice_ptr[U.x + 1] - base) / C);
    const int32_t j0 = U.y < 0 ? 0 : U.y * a.unit_width;
    const int32_t j1 = U.y < 0 ? w : (j0 + a.unit_width < w ? j0 + a.unit_width : w);
    const int64_t p0 = (int64_t)U.x * C + lane * R;
    int32_t L[R];
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        L[r] = __ldcs(a.len + p0 + r);
        acc[r] = 0.0;
    }
    int32_t lmax = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) lmax = L[r] > lmax ? L[r] : lmax;
    const int32_t jend = j1 < lmax ? j1 : lmax;
#pragma unroll 8
    for (int32_t j = j0; j < jend; ++j) {
        const int64_t o = base + (int64_t)j * C + lane * R;
        if constexpr (R == 1) {
            const double v = __ldcs(a.val + o);
            const int32_t c = __ldcs(a.col + o);
            acc[0] = fma(v, ldx(a.x, c), acc[0]);
        } else if constexpr (R == 2) {
            const double2 v = __ldcs(reinterpret_cast<const double2*>(a.val + o));
            const int2 c = __ldcs(reinterpret_cast<const int2*>(a.col + o));
            if (j < L[0]) acc[0] = fma(v.x, ldx(a.x, c.x), acc[0]);
            if (j < L[1]) acc[1] = fma(v.y, ldx(a.x, c.y), acc[1]);
        } else {
            const double2 va = __ldcs(reinterpret_cast<const double2*>(a.val + o));
            const double2 vb = __ldcs(reinterpret_cast<const double2*>(a.val + o + 2));
            const int4 c = __ldcs(reinterpret_cast<const int4*>(a.col + o));
            if (j < L[0]) acc[0] = fma(va.x, ldx(a.x, c.x), acc[0]);
            if (j < L[1]) acc[1] = fma(va.y, ldx(a.x, c.y), acc[1]);
            if (j < L[2]) acc[2] = fma(vb.x, ldx(a.x, c.z), acc[2]);
            if (j < L[3]) acc[3] = fma(vb.y, ldx(a.x, c.w), acc[3]);
        }
    }
    if (U.y < 0) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (p0 + r < a.m) sell_put<MODE>(a, p0 + r, acc[r]);
        return;
    }
    // chunk of a split slice
#pragma unroll
    for (int r = 0; r < R; ++r) a.partial[(int64_t)u * C + lane * R + r] = acc[r];
    __threadfence();
    __syncwarp();
    const int32_t first = u - U.y;
    const int32_t nch = (w + a.unit_width - 1) / a.unit_width;
    unsigned prev = 0;
    if (lane == 0) prev = atomicAdd(a.counters + first, 1u);
    prev = __shfl_sync(kFull, prev, 0);
    if (prev != (unsigned)(nch - 1)) return;
    __threadfence();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        double t = 0.0;
#pragma unroll 8
        for (int32_t c = 0; c < nch; ++c) t += __ldcg(a.partial + (int64_t)(first + c) * C + lane * R + r);
        if (p0 + r < a.m) sell_put<MODE>(a, p0 + r, t);
    }
    __syncwarp();
    if (lane == 0) a.counters[first] = 0u;
}

// ------------------------------------------------------------------- CSR5
//
// A warp processes one tile of S = 32*sigma nonzeros: lane c walks its column
// (nonzeros t*S + c*sigma + r, stored at t*S + r*32 + c, so each step is one
// coalesced 256-byte load) with one DFMA per nonzero.  flags[t*32 + c] bit r
// marks a segment start.  Inside a lane, segments closed by a later flag in the
// same lane are complete; the lane's last segment continues into the following
// lanes up to the next lane holding a flag, which a segmented suffix sum over
// the lanes (shuffles) supplies.
//
// Rows that cross tile boundaries are finished in the same launch: the tile
// where such a row starts stores its open last segment in slot_tail[t0], every
// later tile the row reaches stores its head part in slot_head[t], and each
// takes a ticket on cnt[t0]; the last of the row's tiles to finish adds the
// slots in tile order and writes y (no waiting, deterministic order).  The
// matrix's empty rows are zeroed by the tile warps, a share each.
struct Csr5Args {
    const int32_t* ptr;
    const int32_t* tile_ptr;
    const uint32_t* flags;
    const int32_t* tile_idx;
    const double* tile_val;
    const int32_t* empty_ptr;
    const int32_t* empty_rows;
    double* slot_head;
    double* slot_tail;
    unsigned* cnt;
    const int32_t* zero_rows;
    int32_t n_zero;
    int64_t nnz;
    int64_t ntiles;
    int32_t sigma;
    const double* x;
    double* y;
};

// Contribution of tile t to row r, which spans tiles t0 = ptr[r]/S .. t1;
// the last contributor adds all of them in tile order.  Offsets are int32, so
// the tile numbers come from 32-bit divisions.
__device__ __forceinline__ void csr5_join(const Csr5Args& a, int32_t r, int64_t t, bool tail, double v, uint32_t S) {
    const uint32_t t0 = (uint32_t)a.ptr[r] / S;
    const uint32_t t1 = ((uint32_t)a.ptr[r + 1] - 1u) / S;
    if (tail) a.slot_tail[t] = v;
    else a.slot_head[t] = v;
    // release our slot, acquire the others' (the last ticket sees every slot)
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> ticket(a.cnt[t0]);
    const unsigned prev = ticket.fetch_add(1u, cuda::memory_order_acq_rel);
    if (prev == t1 - t0) {
        double acc = __ldcg(a.slot_tail + t0);
        for (uint32_t u = t0 + 1; u <= t1; ++u) acc += __ldcg(a.slot_head + u);
        ticket.store(0u, cuda::memory_order_relaxed);
        a.y[r] = acc;
    }
}

__device__ __forceinline__ void csr5_tile(const Csr5Args& a, int64_t t, int lane) {
    const int64_t S = 32LL * a.sigma;
    const int64_t base = t * S;
    const uint32_t f = __ldcs(a.flags + t * 32 + lane);
    const int nf = __popc(f);
    // exclusive count of flags in earlier lanes = this lane's first segment index
    int yo = nf;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(kFull, yo, d);
        if (lane >= d) yo += v;
    }
    const int total = __shfl_sync(kFull, yo, 31);  // flagged slots in the tile
    yo -= nf;
    const int32_t row0 = a.tile_ptr[t];
    const int32_t e0 = a.empty_ptr[t], e1 = a.empty_ptr[t + 1];
    const bool listed = e1 > e0;
    const bool cont = a.ptr[row0] != base;  // the tile starts inside row0
    const int64_t kl = base + (int64_t)lane * a.sigma;
    double cur = 0.0, head = 0.0;
    double first = 0.0;  // lane 0: segment 0 when it closes inside the lane
    bool first_join = false;
    int j = 0;  // segments of this lane seen so far
#pragma unroll 8
    for (int r = 0; r < a.sigma; ++r) {
        const int64_t slot = base + (int64_t)r * 32 + lane;
        const bool valid = kl + r < a.nnz;  // false only in the padded last tile
        const double v = valid ? __ldcs(a.tile_val + slot) : 0.0;
        const double xv = valid ? ldx(a.x, __ldcs(a.tile_idx + slot)) : 0.0;
        if ((f >> r) & 1u) {
            if (j == 0) {
                head = cur;
            } else {  // segment yo + j - 1 ends here, complete within the tile
                const int g = yo + j - 1;
                const int32_t row = listed ? a.empty_rows[e0 + g] : row0 + g;
                if (g == 0 && cont) {  // joined after the loop, keeping the loop lean
                    first = cur;
                    first_join = true;
                } else {
                    a.y[row] = cur;
                }
            }
            ++j;
            cur = 0.0;
        }
        cur = fma(v, xv, cur);  // one DFMA per nonzero
    }
    if (nf == 0) head = cur;
    // T_c = head_c + (lane c holds no flag ? T_{c+1} : 0)
    double T = head;
    int stop = nf > 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double Tn = __shfl_down_sync(kFull, T, d);
        const int sn = __shfl_down_sync(kFull, stop, d);
        if (!stop && lane + d < 32) {
            T += Tn;
            stop = sn;
        }
    }
    double next = __shfl_down_sync(kFull, T, 1);
    if (lane == 31) next = 0.0;
    if (first_join) csr5_join(a, row0, t, false, first, (uint32_t)S);
    if (nf > 0) {
        const int g = yo + nf - 1;
        const int32_t row = listed ? a.empty_rows[e0 + g] : row0 + g;
        const double tot = cur + next;
        if (g == 0 && cont) {
            csr5_join(a, row, t, false, tot, (uint32_t)S);  // continues a row begun in an earlier tile
        } else if (g == total - 1 && a.ptr[row + 1] > base + S) {
            csr5_join(a, row, t, true, tot, (uint32_t)S);   // begins here, continues into later tiles
        } else {
            a.y[row] = tot;
        }
    }
    // the matrix's empty rows (y = 0), strided over the tile warps
    for (int64_t z = t * 32 + lane; z < a.n_zero; z += a.ntiles * 32) a.y[a.zero_rows[z]] = 0.0;
}

// Zeroes the empty rows of a matrix without nonzeros (no tiles).
__device__ __forceinline__ void csr5_zero_all(const Csr5Args& a, int64_t i) {
    if (i < a.n_zero) a.y[a.zero_rows[i]] = 0.0;
}

}  // namespace dev
}  // namespace spmv
