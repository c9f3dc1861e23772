// Candidate gather, greedy overlap prune and result compaction.
//
// * gather: per-tile candidate slots written by the fused kernel are packed
//   into one list in tile order (a one-block scan over tile counts, then one
//   block per tile copies) - the order is deterministic.
// * prune: the greedy rule "visit blobs by (radius desc, response desc,
//   row-major position asc); drop a blob when an already kept blob covers more
//   than `overlap` of the smaller circle" equals the lexicographically first
//   maximal independent set of the conflict graph under that priority.  It is
//   computed in parallel: candidates are bucketed in a uniform grid of cells
//   no smaller than the largest possible conflict distance, and every thread
//   repeatedly settles its own candidates: drop if a higher-priority
//   conflicting neighbour is kept, keep once all higher-priority conflicting
//   neighbours are dropped.  The result does not depend on timing or order.
//   The lens overlap is evaluated in FP64 in the same operation order as the
//   CPU oracle (no FMA contraction).
// * output: kept candidates are compacted in list order (per-block counts,
//   a one-block scan, ordered writes) straight into pinned host memory
//   mapped into the device address space.
#include <cstdlib>

#include "internal.h"
#include "prune_common.cuh"

#include <cmath>
#include <vector>

namespace mhfd {

namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ long long block_scan_excl_ll(long long v, long long *sh, long long *tot) {
    // sh: 32 entries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    const long long ex = (warp ? sh[warp - 1] : 0) + x - v;
    *tot = sh[nw - 1];
    __syncthreads();
    return ex;
}

// ---------------------------------------------------------------- gather

// inclusive block scan (kScanThreads threads); *tot gets the block total
__device__ __forceinline__ long long block_scan_incl(long long v, long long *sh, long long *tot) {
    long long tot_;
    const long long ex = block_scan_excl_ll(v, sh, &tot_);
    *tot = tot_;
    return ex + v;
}

// One block: each thread scans a contiguous chunk of tiles serially, one
// block-wide scan joins the chunks.
__global__ void __launch_bounds__(kScanThreads)
    gather_scan(const int *tile_count, int n_tiles, int cap_tile, long long cap, int *tile_off,
                Counters *cnt) {
    __shared__ long long sh[32];
    const int per = (n_tiles + (int)blockDim.x - 1) / (int)blockDim.x;
    const int beg = min(n_tiles, (int)threadIdx.x * per), end = min(n_tiles, beg + per);
    long long loc_s = 0, loc_t = 0;
    for (int t = beg; t < end; ++t) {
        const int c = tile_count[t];
        loc_s += c < cap_tile ? c : cap_tile;
        loc_t += c;
    }
    long long tot_s, tot_t;
    long long run = block_scan_excl_ll(loc_s, sh, &tot_s);
    block_scan_excl_ll(loc_t, sh, &tot_t);
    for (int t = beg; t < end; ++t) {
        tile_off[t] = (int)run;
        const int c = tile_count[t];
        run += c < cap_tile ? c : cap_tile;
    }
    if (threadIdx.x == 0) {
        cnt->n_true = (unsigned long long)tot_t;
        cnt->n_stored = (unsigned long long)(tot_s < cap ? tot_s : cap);
        cnt->overflow = (tot_t > (long long)cnt->n_stored) ? 1 : 0;
        cnt->n_blobs = 0;
        cnt->timeout = cnt->ktimeout;
        cnt->ktimeout = 0;
        cnt->blob_base = 0;
    }
}

__global__ void gather_copy(const int *tile_count, const MhfdCand *stage, int cap_tile,
                            long long cap, const int *tile_off, MhfdCand *cand) {
    const int t = blockIdx.x;
    int m = tile_count[t];
    m = m < cap_tile ? m : cap_tile;
    const long long o = tile_off[t];
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        if (o + k < cap) cand[o + k] = stage[(long long)t * cap_tile + k];
    }
}

// ----------------------------------------------------------------- prune

__global__ void grid_count(const MhfdCand *cand, const Counters *cnt, int cs, int ncx,
                           int *cell_cnt) {
    const long long n = (long long)cnt->n_stored;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const MhfdCand c = cand[j];
        atomicAdd(&cell_cnt[(c.y / cs) * ncx + c.x / cs], 1);
    }
}

// Cell starts (exclusive scan of the counts) in one block: rounds of
// kCellChunk cells are staged in shared memory with coalesced accesses, each
// thread scans a contiguous run of kCellChunk / kScanThreads cells serially
// (the index padded by one word per 32 so that the runs do not share banks)
// and one block scan joins the runs.  The counts are reset to serve as fill
// cursors.
constexpr int kCellChunk = 8192;
__device__ __forceinline__ int cell_pad(int i) { return i + (i >> 5); }

__global__ void __launch_bounds__(kScanThreads)
    grid_scan(int *cell_cnt, int ncells, int *cell_start) {
    __shared__ int sc[kCellChunk + kCellChunk / 32];
    __shared__ long long sh[32];
    constexpr int per = kCellChunk / kScanThreads;
    long long carry = 0;
    for (int base = 0; base < ncells; base += kCellChunk) {
        const int n = min(kCellChunk, ncells - base);
        for (int i = threadIdx.x; i < n; i += blockDim.x) sc[cell_pad(i)] = cell_cnt[base + i];
        __syncthreads();
        const int beg = threadIdx.x * per;
        long long loc = 0;
#pragma unroll
        for (int k = 0; k < per; ++k)
            if (beg + k < n) loc += sc[cell_pad(beg + k)];
        long long tot;
        long long run = carry + block_scan_excl_ll(loc, sh, &tot);
#pragma unroll
        for (int k = 0; k < per; ++k)
            if (beg + k < n) {
                const int v = sc[cell_pad(beg + k)];
                sc[cell_pad(beg + k)] = (int)run;
                run += v;
            }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            cell_start[base + i] = sc[cell_pad(i)];
            cell_cnt[base + i] = 0;  // reused as the fill cursor
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) cell_start[ncells] = (int)carry;
}

__global__ void grid_fill(const MhfdCand *cand, const Counters *cnt, int cs, int ncx,
                          const int *cell_start, int *cursor, int *items, int *state) {
    const long long n = (long long)cnt->n_stored;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const MhfdCand c = cand[j];
        const int cell = (c.y / cs) * ncx + c.x / cs;
        items[cell_start[cell] + atomicAdd(&cursor[cell], 1)] = (int)j;
        state[j] = 0;
    }
}

// Conflict table.  Radii depend only on the scale index and centres sit on
// integer pixels, so whether a kept blob of scale ib overlaps a blob of scale
// ia by more than the threshold depends only on (ib, ia, d2 = dx^2 + dy^2).
// It is evaluated once per detector, for every d2 below the distance where
// the circles separate, with the FP64 lens formula (same operation order as
// the oracle) and stored as bits; the per-pair test in the prune is then
// integer only.  Word w of pair (ib, ia) holds d2 = 32 w .. 32 w + 31.
__global__ void conflict_table_kernel(const double *radius, int nl, const int *lim,
                                      const int *off, double overlap, unsigned *tab) {
    const int pair = blockIdx.y;
    const int ib = pair / nl, ia = pair - ib * nl;
    const int T = lim[pair];
    const int nw = (T + 31) / 32;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        unsigned bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int d2 = 32 * w + b;
            if (d2 >= T) break;
            const double d = __dsqrt_rn((double)d2);
            if (lens_overlap(radius[ib], radius[ia], d) > overlap) bits |= 1u << b;
        }
        tab[off[pair] + w] = bits;
    }
}

__device__ __forceinline__ bool conflict_bit(const MhfdCand &b, const MhfdCand &a,
                                             const ConflictTable &ct) {
    const int dx = a.x - b.x, dy = a.y - b.y;
    const int d2 = dx * dx + dy * dy;
    const int pair = b.i * ct.nl + a.i;
    if (d2 >= __ldg(ct.lim + pair)) return false;
    return (__ldg(ct.tab + __ldg(ct.off + pair) + (d2 >> 5)) >> (d2 & 31)) & 1u;
}

// For candidate j, the higher-priority candidates it conflicts with (overlap
// above the threshold), found once by scanning the 3x3 cells around it.
// Up to kMaxNb are listed; more mark the list as overflowed (-1) and the
// settle loop then rescans the cells instead.
constexpr int kMaxNb = 16;

// One warp per grid cell: the candidates of the cell's 3x3 neighbourhood
// are staged in shared memory once (index and record), then each lane takes
// candidates of the centre cell and tests them against the staged list.  A
// neighbourhood larger than the staging area falls back to reading the
// records from global memory.
constexpr int kCellWarps = 8;
constexpr int kStage = 160;

__device__ __forceinline__ void list_neighbors(int j, const MhfdCand &a, const MhfdCand *cand,
                                               const int *items, int s0, int s1,
                                               const ConflictTable &ct, int W, int *nb_idx,
                                               int &found) {
    for (int p = s0; p < s1; ++p) {
        const int b = items[p];
        if (b == j) continue;
        const MhfdCand cb = cand[b];
        if (!higher(cb, a, W)) continue;
        if (!conflict_bit(cb, a, ct)) continue;
        if (found < kMaxNb) nb_idx[(long long)j * kMaxNb + found] = b;
        ++found;
    }
}

__global__ void __launch_bounds__(32 * kCellWarps)
    prune_neighbors(const MhfdCand *cand, int cs, int ncx, int ncy, const int *cell_start,
                    const int *items, ConflictTable ct, int W, int *nb_idx, int *nb_cnt,
                    int *state) {
    __shared__ MhfdCand s_c[kCellWarps][kStage];
    __shared__ int s_i[kCellWarps][kStage];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncells = ncx * ncy;
    for (int cell = blockIdx.x * kCellWarps + warp; cell < ncells;
         cell += gridDim.x * kCellWarps) {
        const int c0 = cell_start[cell], c1 = cell_start[cell + 1];
        if (c0 == c1) continue;
        const int cy = cell / ncx, cx = cell - cy * ncx;
        const int y0 = max(0, cy - 1), y1 = min(ncy - 1, cy + 1);
        const int x0 = max(0, cx - 1), x1 = min(ncx - 1, cx + 1);
        int m = 0;
        for (int gy = y0; gy <= y1; ++gy) {
            // the three cells of a grid row are contiguous in `items`
            const int s0 = cell_start[gy * ncx + x0], s1 = cell_start[gy * ncx + x1 + 1];
            for (int p = s0 + lane; p < s1; p += 32) {
                const int q = m + (p - s0);
                if (q < kStage) {
                    const int b = items[p];
                    s_i[warp][q] = b;
                    s_c[warp][q] = cand[b];
                }
            }
            m += s1 - s0;
        }
        __syncwarp();
        for (int p = c0 + lane; p < c1; p += 32) {
            const int j = items[p];
            const MhfdCand a = cand[j];
            int found = 0;
            if (m <= kStage) {
                for (int q = 0; q < m; ++q) {
                    const int b = s_i[warp][q];
                    if (b == j) continue;
                    const MhfdCand cb = s_c[warp][q];
                    if (!higher(cb, a, W)) continue;
                    if (!conflict_bit(cb, a, ct)) continue;
                    if (found < kMaxNb) nb_idx[(long long)j * kMaxNb + found] = b;
                    ++found;
                }
            } else {
                for (int gy = y0; gy <= y1; ++gy)
                    list_neighbors(j, a, cand, items, cell_start[gy * ncx + x0],
                                   cell_start[gy * ncx + x1 + 1], ct, W, nb_idx, found);
            }
            nb_cnt[j] = found <= kMaxNb ? found : -1;
            state[j] = found == 0 ? 1 : 0;
        }
        __syncwarp();
    }
}

// 0 = undecided, 1 = kept, 2 = dropped
__device__ int settle(int j, const MhfdCand *cand, int cs, int ncx, int ncy,
                      const int *cell_start, const int *items, const ConflictTable &ct, int W,
                      const int *nb_idx, const int *nb_cnt, const volatile int *state) {
    const int m = nb_cnt[j];
    if (m >= 0) {
        bool waiting = false;
        for (int q = 0; q < m; ++q) {
            const int s = state[nb_idx[(long long)j * kMaxNb + q]];
            if (s == 1) return 2;
            if (s == 0) waiting = true;
        }
        return waiting ? 0 : 1;
    }
    const MhfdCand a = cand[j];
    const int cx = a.x / cs, cy = a.y / cs;
    bool waiting = false;
    for (int gy = max(0, cy - 1); gy <= min(ncy - 1, cy + 1); ++gy)
        for (int gx = max(0, cx - 1); gx <= min(ncx - 1, cx + 1); ++gx) {
            const int c = gy * ncx + gx;
            for (int p = cell_start[c]; p < cell_start[c + 1]; ++p) {
                const int b = items[p];
                if (b == j) continue;
                const MhfdCand cb = cand[b];
                if (!higher(cb, a, W)) continue;
                const int s = state[b];
                if (s == 2) continue;
                if (!conflict_bit(cb, a, ct)) continue;
                if (s == 1) return 2;
                waiting = true;
            }
        }
    return waiting ? 0 : 1;
}

__global__ void __launch_bounds__(256)
    lfmis_kernel(const MhfdCand *cand, Counters *cnt, int cs, int ncx, int ncy,
                 const int *cell_start, const int *items, ConflictTable ct, int W,
                 const int *nb_idx, const int *nb_cnt, int *state, long long max_sweeps,
                 unsigned long long max_ns) {
    // Every thread settles its own candidates; a candidate waits only on
    // higher-priority ones, so the highest undecided candidate can always be
    // settled and the sweeps end.  The waits are bounded in count and time;
    // on expiry the detection reports MHFD_ERR_TIMEOUT instead of spinning.
    const long long n = (long long)cnt->n_stored;
    volatile int *vs = state;
    const long long g0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long gs = (long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = globaltimer_ns();
    long long sweep = 0;
    bool pending = true;
    for (; sweep < max_sweeps; ++sweep) {
        pending = false;
        for (long long j = g0; j < n; j += gs) {
            if (vs[j] != 0) continue;
            const int r = settle((int)j, cand, cs, ncx, ncy, cell_start, items, ct, W, nb_idx,
                                 nb_cnt, vs);
            if (r == 0)
                pending = true;
            else
                vs[j] = r;
        }
        if (!pending) break;
        __nanosleep(100);
        if ((sweep & 63) == 63 && globaltimer_ns() - t0 > max_ns) break;
    }
    if (pending) atomicOr(&cnt->timeout, 1);
}

__global__ void keep_all(const Counters *cnt, int *state) {
    const long long n = (long long)cnt->n_stored;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        state[j] = 1;
}

// ---------------------------------------------------------------- output

struct DevAcc {
    int per_scale[64];
};

__global__ void __launch_bounds__(256)
    out_count(const MhfdCand *cand, const int *state, const Counters *cnt, int *block_cnt,
              double *block_sum) {
    __shared__ long long shc[256];
    __shared__ double shs[256];
    const long long n = (long long)cnt->n_stored;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long beg = min(n, (long long)blockIdx.x * per), end = min(n, beg + per);
    long long c = 0;
    double s = 0.0;
    for (long long j = beg + threadIdx.x; j < end; j += blockDim.x)
        if (state[j] == 1) {
            ++c;
            s += (double)cand[j].resp;
        }
    shc[threadIdx.x] = c;
    shs[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {  // fixed-order tree: deterministic sum
        if ((int)threadIdx.x < o) {
            shc[threadIdx.x] += shc[threadIdx.x + o];
            shs[threadIdx.x] += shs[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        block_cnt[blockIdx.x] = (int)shc[0];
        block_sum[blockIdx.x] = shs[0];
    }
}

// nb = 256 blocks: one thread per block count; the response sum is added in
// block order by a fixed tree (deterministic)
__global__ void __launch_bounds__(256)
    out_scan(int *block_cnt, const double *block_sum, int nb, Counters *cnt, double *sum_out,
             int *per_scale, unsigned long long *arena, unsigned long long arena_cap) {
    __shared__ long long sh[32];
    __shared__ double ss[256];
    const int b = threadIdx.x;
    const long long v = b < nb ? block_cnt[b] : 0;
    ss[b] = b < nb ? block_sum[b] : 0.0;
    long long tot;
    const long long ex = block_scan_excl_ll(v, sh, &tot);
    if (b < nb) block_cnt[b] = (int)ex;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (b < o) ss[b] += ss[b + o];
        __syncthreads();
    }
    if (b == 0) {
        unsigned long long n = (unsigned long long)tot, base = 0;
        if (arena) {
            base = atomicAdd(arena, n);
            if (base >= arena_cap) {
                n = 0;
                cnt->overflow = 1;
            } else if (base + n > arena_cap) {
                n = arena_cap - base;
                cnt->overflow = 1;
            }
        }
        cnt->blob_base = base;
        cnt->n_blobs = n;
        *sum_out = ss[0];
    }
    if (b < 64) per_scale[b] = 0;
}

__global__ void __launch_bounds__(256)
    out_write(const MhfdCand *cand, const int *state, const Counters *cnt, const int *block_off,
              const float *sigma, const float *radius_f, mhfd_blob *blobs, mhfd_blob *cands,
              int *per_scale) {
    __shared__ int sh_scale[64];
    __shared__ int sh_w[8];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) sh_scale[i] = 0;
    __syncthreads();
    const long long n = (long long)cnt->n_stored;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long beg = min(n, (long long)blockIdx.x * per), end = min(n, beg + per);
    const long long obase = (long long)cnt->blob_base, lim = (long long)cnt->n_blobs;
    long long out = block_off[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = beg; base < end; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        const bool valid = j < end;
        MhfdCand c;
        c.x = c.y = c.i = 0;
        c.resp = 0.0f;
        int keep = 0;
        if (valid) {
            c = cand[j];
            keep = state[j] == 1;
            if (cands) {
                mhfd_blob b;
                b.x = c.x;
                b.y = c.y;
                b.scale_idx = c.i;
                b.sigma = sigma[c.i];
                b.radius = radius_f[c.i];
                b.response = c.resp;
                cands[j] = b;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) sh_w[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += sh_w[w];
            total += sh_w[w];
        }
        const long long pos = out + before + __popc(bal & ((1u << lane) - 1u));
        if (keep && pos < lim) {
            mhfd_blob b;
            b.x = c.x;
            b.y = c.y;
            b.scale_idx = c.i;
            b.sigma = sigma[c.i];
            b.radius = radius_f[c.i];
            b.response = c.resp;
            blobs[obase + pos] = b;
            atomicAdd(&sh_scale[c.i & 63], 1);
        }
        out += total;
        __syncthreads();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (sh_scale[i]) atomicAdd(&per_scale[i], sh_scale[i]);
}

__global__ void out_publish(const Counters *cnt, const double *sum, const int *per_scale,
                            const MhfdStretch *st, HostResult *h) {
    const int t = threadIdx.x;
    if (t < 64) h->per_scale[t] = per_scale[t];
    if (t == 0) {
        h->c = *cnt;
        h->sum_resp = *sum;
        h->lo = st ? st->lo : 0.0f;
        h->hi = st ? st->hi : 0.0f;
    }
}

// Positions and scale indices are clamped into the image and the ladder so
// that a malformed list cannot address memory outside the prune grid.
__global__ void pack_kernel(const int32_t *x, const int32_t *y, const int32_t *i, const float *r,
                            long long n, int H, int W, int n_levels, MhfdCand *cand,
                            Counters *cnt) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        MhfdCand c;
        c.x = min(max(x[j], 0), W - 1);
        c.y = min(max(y[j], 0), H - 1);
        c.i = min(max(i[j], 0), n_levels - 1);
        c.resp = r[j];
        cand[j] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cnt->n_true = cnt->n_stored = (unsigned long long)n;
        cnt->overflow = 0;
        cnt->timeout = 0;
        cnt->n_blobs = 0;
    }
}

__global__ void keep_kernel(const int *state, const Counters *cnt, long long n, int prune_on,
                            uint8_t *keep) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        keep[j] = prune_on ? (state[j] == 1 ? 1 : 0) : 1;
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

int enqueue_gather(const int *tile_count, const MhfdCand *stage, int n_tiles, int cap_tile,
                   long long cap, int *tile_off, MhfdCand *cand, Counters *cnt, cudaStream_t s) {
    gather_scan<<<1, kScanThreads, 0, s>>>(tile_count, n_tiles, cap_tile, cap, tile_off, cnt);
    gather_copy<<<n_tiles, 128, 0, s>>>(tile_count, stage, cap_tile, cap, tile_off, cand);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int build_conflict_table(const double *d_radius, const std::vector<double> &radius,
                         double overlap, ConflictTable *ct) {
    const int nl = (int)radius.size();
    std::vector<int> lim(nl * nl, 0), off(nl * nl, 0);
    int words = 0;
    for (int ib = 0; ib < nl; ++ib)
        for (int ia = 0; ia < nl; ++ia) {
            const int pair = ib * nl + ia;
            off[pair] = words;
            if (ib < ia) continue;  // a kept, higher-priority blob never has a smaller scale
            const double rs = radius[ib] + radius[ia];
            lim[pair] = (int)std::ceil(rs * rs) + 2;  // overlap is 0 from here on
            words += (lim[pair] + 31) / 32;
        }
    ct->nl = nl;
    int *d_lim = nullptr, *d_off = nullptr;
    unsigned *d_tab = nullptr;
    MHFD_CUDA(cudaMalloc(&d_lim, sizeof(int) * nl * nl));
    MHFD_CUDA(cudaMalloc(&d_off, sizeof(int) * nl * nl));
    MHFD_CUDA(cudaMalloc(&d_tab, sizeof(unsigned) * (words > 0 ? words : 1)));
    ct->lim = d_lim;
    ct->off = d_off;
    ct->tab = d_tab;
    ct->bytes = sizeof(int) * 2 * nl * nl + sizeof(unsigned) * (words > 0 ? words : 1);
    MHFD_CUDA(cudaMemcpy(d_lim, lim.data(), sizeof(int) * nl * nl, cudaMemcpyHostToDevice));
    MHFD_CUDA(cudaMemcpy(d_off, off.data(), sizeof(int) * nl * nl, cudaMemcpyHostToDevice));
    conflict_table_kernel<<<dim3(8, nl * nl), 128>>>(d_radius, nl, d_lim, d_off, overlap, d_tab);
    MHFD_CUDA(cudaGetLastError());
    MHFD_CUDA(cudaDeviceSynchronize());
    return MHFD_OK;
}

void free_conflict_table(ConflictTable *ct) {
    if (ct->lim) cudaFree((void *)ct->lim);
    if (ct->off) cudaFree((void *)ct->off);
    if (ct->tab) cudaFree((void *)ct->tab);
    ct->lim = ct->off = nullptr;
    ct->tab = nullptr;
}

int enqueue_prune(const MhfdCand *cand, const Counters *cnt_c, long long cap, int H, int W,
                  const ConflictTable &ct, double radius_max, double overlap, PruneBuffers *pb,
                  cudaStream_t s) {
    (void)cap;
    Counters *cnt = const_cast<Counters *>(cnt_c);
    if (overlap >= 1.0) {
        keep_all<<<sm_count() * 4, 256, 0, s>>>(cnt, pb->state);
        MHFD_CUDA(cudaGetLastError());
        return MHFD_OK;
    }
    // cell edge >= the largest conflict distance r1 + r2 <= 2 * radius_max
    const int cs = (int)ceil(2.0 * radius_max) + 1;
    const int ncx = (W + cs - 1) / cs, ncy = (H + cs - 1) / cs;
    const int ncells = ncx * ncy;
    if ((size_t)ncells + 1 > pb->ncells_cap) return fail(MHFD_ERR_INVALID_ARG, "prune grid too large");
    MHFD_CUDA(cudaMemsetAsync(pb->cell_cnt, 0, sizeof(int) * (ncells + 1), s));
    const int sms = sm_count();
    grid_count<<<sms * 4, 256, 0, s>>>(cand, cnt, cs, ncx, pb->cell_cnt);
    grid_scan<<<1, kScanThreads, 0, s>>>(pb->cell_cnt, ncells, pb->cell_start);
    grid_fill<<<sms * 4, 256, 0, s>>>(cand, cnt, cs, ncx, pb->cell_start, pb->cell_cnt,
                                      pb->cell_items, pb->state);
    {
        const int ncells_all = ncx * ncy;
        int blocks = (ncells_all + kCellWarps - 1) / kCellWarps;
        if (blocks > sms * 16) blocks = sms * 16;
        prune_neighbors<<<blocks, 32 * kCellWarps, 0, s>>>(cand, cs, ncx, ncy, pb->cell_start,
                                                           pb->cell_items, ct, W, pb->nb_idx,
                                                           pb->nb_cnt, pb->state);
    }
    MHFD_CUDA(cudaGetLastError());
    int per_sm = 0;
    MHFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lfmis_kernel, 256, 0));
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * (per_sm < 4 ? per_sm : 4);
    long long max_sweeps = 1ll << 24;
    unsigned long long max_ns = 2000000000ull;  // 2 s of device time
    // MHFD_PRUNE_MAX_SWEEPS: a smaller bound on the settle loop, for tests of
    // the timeout report (0 gives up before the first sweep)
    if (const char *e = std::getenv("MHFD_PRUNE_MAX_SWEEPS")) {
        if (*e) max_sweeps = std::atoll(e) < 0 ? 0 : std::atoll(e);
    }
    ConflictTable ctv = ct;
    void *args[] = {(void *)&cand, (void *)&cnt, (void *)&cs, (void *)&ncx, (void *)&ncy,
                    (void *)&pb->cell_start, (void *)&pb->cell_items, (void *)&ctv, (void *)&W,
                    (void *)&pb->nb_idx, (void *)&pb->nb_cnt, (void *)&pb->state,
                    (void *)&max_sweeps, (void *)&max_ns};
    // the settle loop needs all its blocks resident: a cooperative launch
    // guarantees it; inside a stream capture (graphs) a plain launch of a
    // grid that fits the GPU is used, and its bounded waits turn any
    // non-resident block into a reported timeout rather than a hang
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    MHFD_CUDA(cudaStreamIsCapturing(s, &capst));
    if (capst == cudaStreamCaptureStatusActive) {
        lfmis_kernel<<<grid, 256, 0, s>>>(cand, cnt, cs, ncx, ncy, pb->cell_start, pb->cell_items,
                                          ctv, W, pb->nb_idx, pb->nb_cnt, pb->state, max_sweeps,
                                          max_ns);
        MHFD_CUDA(cudaGetLastError());
    } else {
        MHFD_CUDA(cudaLaunchCooperativeKernel((const void *)lfmis_kernel, grid, 256, args, 0, s));
    }
    return MHFD_OK;
}

int enqueue_output(const MhfdCand *cand, const int *state, const Counters *cnt_c, long long cap,
                   const float *d_sigma, const float *d_radius_f, int prune_on,
                   HostResult *h_res_dev, mhfd_blob *h_blobs_dev, mhfd_blob *h_cands_dev,
                   const MhfdStretch *st, int *block_tmp, double *block_sum,
                   unsigned long long *arena, unsigned long long arena_cap, cudaStream_t s) {
    (void)cap;
    (void)prune_on;
    Counters *cnt = const_cast<Counters *>(cnt_c);
    const int nb = 256;
    // block_tmp: nb block counts followed by 64 per-scale counters
    int *per_scale = block_tmp + nb;
    double *sum = block_sum + nb;
    out_count<<<nb, 256, 0, s>>>(cand, state, cnt, block_tmp, block_sum);
    out_scan<<<1, 256, 0, s>>>(block_tmp, block_sum, nb, cnt, sum, per_scale, arena, arena_cap);
    out_write<<<nb, 256, 0, s>>>(cand, state, cnt, block_tmp, d_sigma, d_radius_f, h_blobs_dev,
                                 h_cands_dev, per_scale);
    out_publish<<<1, 64, 0, s>>>(cnt, sum, per_scale, st, h_res_dev);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int enqueue_pack(const int32_t *x, const int32_t *y, const int32_t *i, const float *r,
                 long long n, int H, int W, int n_levels, MhfdCand *cand, Counters *cnt,
                 cudaStream_t s) {
    pack_kernel<<<sm_count() * 2, 256, 0, s>>>(x, y, i, r, n, H, W, n_levels, cand, cnt);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int enqueue_keep(const int *state, const Counters *cnt, long long n, int prune_on, uint8_t *keep,
                 cudaStream_t s) {
    keep_kernel<<<sm_count() * 2, 256, 0, s>>>(state, cnt, n, prune_on, keep);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

}  // namespace mhfd
