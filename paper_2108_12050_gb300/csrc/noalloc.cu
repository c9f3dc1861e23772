// Allocation-free overlap prune (mhfd_prune_noalloc).
//
// Some callers cannot allocate device memory at all: code running where the
// CUDA allocator is off limits (a host callback or a real-time thread that
// must not block on cudaMalloc's implicit synchronisation, an embedding
// framework that owns every allocation, an instrument controller with a fixed
// memory budget).  For them this file offers the overlap prune without a
// detector and without any cudaMalloc/cudaFree: all of its working memory
// lives in one file-scope device array of fixed size, which every GPU that
// loads this library keeps until the process exits.
//
// Limits: at most kMaxCand candidates, at most kMaxCells cells of the
// neighbour grid (cells are about 2 r_max pixels square), at most 64 scale
// indices.  Larger calls are rejected with MHFD_ERR_INVALID_ARG.
//
// Every call uses the same array and leaves its contents behind; each call
// clears what must start at zero.  Calls whose work overlaps on the GPU (for
// example on two streams) race on the array and must be serialised by the
// caller.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call
// before any stream capture.  The address is kept for the process's life, so
// cudaDeviceReset after the first call is not supported.
//
// The settle loop's wait is bounded (2^24 sweeps or 2 s of device time, or
// MHFD_PRUNE_MAX_SWEEPS sweeps); candidates it leaves unresolved when the
// bound runs out get keep = 2, so the caller sees an incomplete result.
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>

#include "internal.h"
#include "prune_common.cuh"

namespace mhfd {

namespace {

constexpr long long kMaxCand = 65536;
constexpr long long kMaxCells = 65536;
constexpr int kMaxNbNa = 16;
constexpr int kMaxDevices = 64;

// byte layout of the scratch array
constexpr size_t kOffCand = 0;                                          // MhfdCand[kMaxCand]
constexpr size_t kOffItems = kOffCand + 16 * kMaxCand;                  // int[kMaxCand]
constexpr size_t kOffState = kOffItems + 4 * kMaxCand;                  // int[kMaxCand]
constexpr size_t kOffNbCnt = kOffState + 4 * kMaxCand;                  // int[kMaxCand]
constexpr size_t kOffNbIdx = kOffNbCnt + 4 * kMaxCand;                  // int[kMaxCand * 16]
constexpr size_t kOffCellCnt = kOffNbIdx + 4 * kMaxNbNa * kMaxCand;     // int[kMaxCells + 1]
constexpr size_t kOffCellStart = kOffCellCnt + 4 * (kMaxCells + 1);     // int[kMaxCells + 1]
constexpr size_t kOffFlags = kOffCellStart + 4 * (kMaxCells + 1);       // int[64]
constexpr size_t kScratchBytes = ((kOffFlags + 256 + 255) / 256) * 256;  // ~6.6 MB

__device__ __align__(256) unsigned char g_prune_scratch[kScratchBytes];

struct Radii {
    double r[64];
};

struct Scratch {
    MhfdCand *cand;
    int *items, *state, *nb_cnt, *nb_idx, *cell_cnt, *cell_start, *flags;
};

Scratch carve(unsigned char *base) {
    Scratch s;
    s.cand = reinterpret_cast<MhfdCand *>(base + kOffCand);
    s.items = reinterpret_cast<int *>(base + kOffItems);
    s.state = reinterpret_cast<int *>(base + kOffState);
    s.nb_cnt = reinterpret_cast<int *>(base + kOffNbCnt);
    s.nb_idx = reinterpret_cast<int *>(base + kOffNbIdx);
    s.cell_cnt = reinterpret_cast<int *>(base + kOffCellCnt);
    s.cell_start = reinterpret_cast<int *>(base + kOffCellStart);
    s.flags = reinterpret_cast<int *>(base + kOffFlags);
    return s;
}

__global__ void na_pack(const int32_t *x, const int32_t *y, const int32_t *i, const float *r,
                        int n, int H, int W, int nl, int cs, int ncx, Scratch s) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        MhfdCand c;
        c.x = min(max(x[j], 0), W - 1);
        c.y = min(max(y[j], 0), H - 1);
        c.i = min(max(i[j], 0), nl - 1);
        c.resp = r[j];
        s.cand[j] = c;
        s.state[j] = 0;
        atomicAdd(&s.cell_cnt[(c.y / cs) * ncx + c.x / cs], 1);
    }
}

// exclusive scan of the cell counts by one block of 1024 threads (tiled)
__global__ void __launch_bounds__(1024) na_scan(int ncells, Scratch s) {
    __shared__ int sh[32];
    int carry = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < ncells; base += 1024) {
        const int c = base + threadIdx.x;
        const int v = c < ncells ? s.cell_cnt[c] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) sh[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = sh[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            sh[lane] = w;
        }
        __syncthreads();
        const int ex = (warp ? sh[warp - 1] : 0) + x - v;
        if (c < ncells) {
            s.cell_start[c] = carry + ex;
            s.cell_cnt[c] = 0;  // becomes the fill cursor
        }
        carry += sh[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) s.cell_start[ncells] = carry;
}

__global__ void na_fill(int n, int cs, int ncx, Scratch s) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const MhfdCand c = s.cand[j];
        const int cell = (c.y / cs) * ncx + c.x / cs;
        s.items[s.cell_start[cell] + atomicAdd(&s.cell_cnt[cell], 1)] = j;
    }
}

__device__ __forceinline__ bool na_conflict(const MhfdCand &b, const MhfdCand &a,
                                            const Radii &rad, double overlap) {
    const double dx = (double)(a.x - b.x), dy = (double)(a.y - b.y);
    const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    return lens_overlap(rad.r[b.i], rad.r[a.i], d) > overlap;
}

__global__ void __launch_bounds__(256)
    na_neighbors(int n, int cs, int ncx, int ncy, int W, const Radii rad, double overlap,
                 Scratch s) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const MhfdCand a = s.cand[j];
        const int cx = a.x / cs, cy = a.y / cs;
        int found = 0;
        for (int gy = max(0, cy - 1); gy <= min(ncy - 1, cy + 1); ++gy)
            for (int gx = max(0, cx - 1); gx <= min(ncx - 1, cx + 1); ++gx) {
                const int c = gy * ncx + gx;
                for (int p = s.cell_start[c]; p < s.cell_start[c + 1]; ++p) {
                    const int b = s.items[p];
                    if (b == j) continue;
                    const MhfdCand cb = s.cand[b];
                    if (!higher(cb, a, W) || !na_conflict(cb, a, rad, overlap)) continue;
                    if (found < kMaxNbNa) s.nb_idx[j * kMaxNbNa + found] = b;
                    ++found;
                }
            }
        s.nb_cnt[j] = found <= kMaxNbNa ? found : -1;
        if (found == 0) s.state[j] = 1;
    }
}

__device__ int na_settle(int j, int cs, int ncx, int ncy, int W, const Radii &rad,
                         double overlap, const Scratch &s, const volatile int *state) {
    const int m = s.nb_cnt[j];
    if (m >= 0) {
        bool waiting = false;
        for (int q = 0; q < m; ++q) {
            const int st = state[s.nb_idx[j * kMaxNbNa + q]];
            if (st == 1) return 2;
            if (st == 0) waiting = true;
        }
        return waiting ? 0 : 1;
    }
    const MhfdCand a = s.cand[j];
    const int cx = a.x / cs, cy = a.y / cs;
    bool waiting = false;
    for (int gy = max(0, cy - 1); gy <= min(ncy - 1, cy + 1); ++gy)
        for (int gx = max(0, cx - 1); gx <= min(ncx - 1, cx + 1); ++gx) {
            const int c = gy * ncx + gx;
            for (int p = s.cell_start[c]; p < s.cell_start[c + 1]; ++p) {
                const int b = s.items[p];
                if (b == j) continue;
                const MhfdCand cb = s.cand[b];
                if (!higher(cb, a, W)) continue;
                const int st = state[b];
                if (st == 2 || !na_conflict(cb, a, rad, overlap)) continue;
                if (st == 1) return 2;
                waiting = true;
            }
        }
    return waiting ? 0 : 1;
}

// Same settling rule as the detector's prune; waits bounded in sweeps and in
// device time, flags[0] = 1 on expiry.
__global__ void __launch_bounds__(256)
    na_settle_all(int n, int cs, int ncx, int ncy, int W, const Radii rad, double overlap,
                  Scratch s, long long max_sweeps, unsigned long long max_ns) {
    volatile int *vs = s.state;
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    const unsigned long long t0 = globaltimer_ns();
    bool pending = true;
    for (long long sweep = 0; sweep < max_sweeps; ++sweep) {
        pending = false;
        for (int j = g0; j < n; j += gs) {
            if (vs[j] != 0) continue;
            const int r = na_settle(j, cs, ncx, ncy, W, rad, overlap, s, vs);
            if (r == 0)
                pending = true;
            else
                vs[j] = r;
        }
        if (!pending) break;
        __nanosleep(100);
        if ((sweep & 63) == 63 && globaltimer_ns() - t0 > max_ns) break;
    }
    if (pending) atomicExch(&s.flags[0], 1);
}

// keep: 1 kept, 0 dropped, 2 left unresolved by a settle loop that gave up
// (state 0 survives the loop only when its bound ran out)
__global__ void na_keep(int n, Scratch s, uint8_t *keep) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int st = s.state[j];
        keep[j] = st == 1 ? 1 : (st == 0 ? 2 : 0);
    }
}

std::mutex g_na_mu;
unsigned char *g_na_base[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_base(unsigned char **out) {
    int dev = 0;
    MHFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(MHFD_ERR_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_base[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_prune_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_prune_scratch)");
        g_na_base[dev] = reinterpret_cast<unsigned char *>(p);
    }
    *out = g_na_base[dev];
    return MHFD_OK;
}

}  // namespace

}  // namespace mhfd

using namespace mhfd;

extern "C" int mhfd_prune_noalloc(const double *radius, int32_t n_levels, float overlap,
                                  const int32_t *d_x, const int32_t *d_y, const int32_t *d_i,
                                  const float *d_resp, int64_t n_cand, int32_t H, int32_t W,
                                  uint8_t *d_keep, void *stream) {
    if (!radius || !d_x || !d_y || !d_i || !d_resp || !d_keep)
        return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    if (n_levels < 1 || n_levels > 64) return fail(MHFD_ERR_INVALID_ARG, "n_levels must be in [1, 64]");
    if (!(overlap >= 0.0f)) return fail(MHFD_ERR_INVALID_ARG, "overlap must be >= 0");
    if (H < 1 || W < 1) return fail(MHFD_ERR_INVALID_ARG, "H and W must be >= 1");
    if (n_cand < 0 || n_cand > kMaxCand)
        return fail(MHFD_ERR_INVALID_ARG, "n_cand exceeds the fixed scratch limit of " +
                                              std::to_string(kMaxCand) + " candidates");
    Radii rad;
    double rmax = 0.0;
    for (int l = 0; l < 64; ++l) rad.r[l] = 0.0;
    for (int l = 0; l < n_levels; ++l) {
        if (!(radius[l] > 0.0) || !std::isfinite(radius[l]))
            return fail(MHFD_ERR_INVALID_ARG, "radii must be positive and finite");
        rad.r[l] = radius[l];
        rmax = radius[l] > rmax ? radius[l] : rmax;
    }
    const int cs = (int)std::ceil(2.0 * rmax) + 1;
    const long long ncx = (W + cs - 1) / cs, ncy = (H + cs - 1) / cs;
    if (ncx * ncy > kMaxCells)
        return fail(MHFD_ERR_INVALID_ARG, "image needs " + std::to_string(ncx * ncy) +
                                              " grid cells; the fixed scratch holds " +
                                              std::to_string(kMaxCells));
    unsigned char *base = nullptr;
    int rc = scratch_base(&base);
    if (rc) return rc;
    if (n_cand == 0) return MHFD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const Scratch sc = carve(base);
    const int n = (int)n_cand, ncells = (int)(ncx * ncy);
    // clear what must start at zero: the cell counters and the timeout flag
    MHFD_CUDA(cudaMemsetAsync(sc.cell_cnt, 0, sizeof(int) * (ncells + 1), s));
    MHFD_CUDA(cudaMemsetAsync(sc.flags, 0, sizeof(int) * 64, s));
    int dev = 0, sms = 1;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 4;
    na_pack<<<grid, 256, 0, s>>>(d_x, d_y, d_i, d_resp, n, H, W, n_levels, cs, (int)ncx, sc);
    na_scan<<<1, 1024, 0, s>>>(ncells, sc);
    na_fill<<<grid, 256, 0, s>>>(n, cs, (int)ncx, sc);
    const double ov = (double)overlap;
    const int icx = (int)ncx, icy = (int)ncy;
    na_neighbors<<<grid, 256, 0, s>>>(n, cs, icx, icy, W, rad, ov, sc);
    MHFD_CUDA(cudaGetLastError());
    int per_sm = 0;
    MHFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, na_settle_all, 256, 0));
    if (per_sm < 1) per_sm = 1;
    const int cgrid = sms * (per_sm < 4 ? per_sm : 4);
    long long max_sweeps = 1ll << 24;
    unsigned long long max_ns = 2000000000ull;
    // MHFD_PRUNE_MAX_SWEEPS: a smaller bound on the settle loop, as for the
    // detector's prune (0 gives up before the first sweep)
    if (const char *e = std::getenv("MHFD_PRUNE_MAX_SWEEPS")) {
        if (*e) max_sweeps = std::atoll(e) < 0 ? 0 : std::atoll(e);
    }
    Scratch scv = sc;
    Radii radv = rad;
    double ovv = ov;
    int nn = n, csv = cs, Wv = W;
    void *args[] = {(void *)&nn, (void *)&csv, (void *)&icx, (void *)&icy, (void *)&Wv,
                    (void *)&radv, (void *)&ovv, (void *)&scv, (void *)&max_sweeps,
                    (void *)&max_ns};
    MHFD_CUDA(cudaLaunchCooperativeKernel((const void *)na_settle_all, cgrid, 256, args, 0, s));
    na_keep<<<grid, 256, 0, s>>>(n, sc, d_keep);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}
