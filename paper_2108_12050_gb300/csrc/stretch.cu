// Histogram stretch bounds of §3 on the device: the k-th and (N-1-k)-th
// smallest pixel values found exactly by an MSD radix select over 8-bit
// digits (1 pass for uint8, 2 for uint16, 4 for float32 keys), entirely on
// the stream (no host round trip).  Each pass builds, per target, the digit
// histogram of the pixels whose higher digits match the target's prefix in
// shared memory (runs of equal digits counted in registers first; the
// histogram replicated per lane group so that the few hot digits of an image
// do not serialise the block's atomics); a one-block select kernel then
// picks the digit that contains the remaining rank.
#include "internal.h"

namespace mhfd {

namespace {

__device__ __forceinline__ unsigned key_u8(unsigned char v) { return v; }
__device__ __forceinline__ unsigned key_u16(unsigned short v) { return v; }
// order-preserving map of float bits onto unsigned integers
__device__ __forceinline__ unsigned key_f32(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unkey_f32(unsigned k) {
    const unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

__global__ void sel_init(SelState *sel, unsigned long long k, unsigned long long n) {
    const int t = threadIdx.x;
    if (t == 0) {
        sel->prefix[0] = sel->prefix[1] = 0;
        sel->rank[0] = k;
        sel->rank[1] = n - 1 - k;
    }
    for (int i = t; i < 512; i += blockDim.x) (&sel->hist[0][0])[i] = 0;
}

template <int DT>
__device__ __forceinline__ unsigned load_key(const char *row, int x) {
    if (DT == 0) return key_u8(__ldg(reinterpret_cast<const unsigned char *>(row) + x));
    if (DT == 1) return key_u16(__ldg(reinterpret_cast<const unsigned short *>(row) + x));
    return key_f32(__ldg(reinterpret_cast<const float *>(row) + x));
}

// One pass of the select (BITS = key width).  Rows are spread over blocks;
// each thread reads VEC consecutive pixels of a row per step (one 16-byte
// load when the image is 16-byte aligned) and aggregates runs of equal
// digits in registers before adding them to the block's shared histograms,
// which are merged into the global histograms at the end.
// shared histograms of one block: [target][replica][digit], a replica per
// group of lanes (lane % kRep), rows padded to spread the replicas' banks
constexpr int kRep = 8;
constexpr int kRow = 257;
struct HistSmem {
    unsigned v[2][kRep][kRow];
};

struct RunAcc {
    unsigned cur = 0xffffffffu, n = 0;
    __device__ __forceinline__ void add(unsigned d, unsigned *h) {
        if (d == cur) {
            ++n;
        } else {
            if (n) atomicAdd(&h[cur], n);
            cur = d;
            n = 1;
        }
    }
    __device__ __forceinline__ void flush(unsigned *h) {
        if (n) atomicAdd(&h[cur], n);
        n = 0;
    }
};

// Histogram accumulation of one pass over rows [y0, H) step ystep of one
// image into the block's shared histograms.
template <int DT, int BITS, bool FIRST>
__device__ __forceinline__ void hist_rows_p(const char *img, int H, int W, long long pitch,
                                            int pass, const SelState *sel, int y0, int ystep,
                                            HistSmem *hs) {
    unsigned *h[2] = {hs->v[0][threadIdx.x % kRep], hs->v[1][threadIdx.x % kRep]};
    constexpr int ES = DT == 0 ? 1 : (DT == 1 ? 2 : 4);
    constexpr int VEC = 16 / ES;
    constexpr bool first = FIRST;  // the first pass counts every pixel for both targets
    const int shift = FIRST ? BITS - 8 : BITS - 8 * (pass + 1);
    const unsigned p0 = sel->prefix[0], p1 = sel->prefix[1];
    const bool vec_ok = ((reinterpret_cast<unsigned long long>(img) | (unsigned long long)pitch) & 15ull) == 0;
    RunAcc r0, r1;
    auto take = [&](unsigned key) {
        const unsigned digit = (key >> shift) & 0xffu;
        const unsigned hi = first ? 0u : (key >> (shift + 8));
        if (first || hi == p0) r0.add(digit, h[0]);
        if (!first && hi == p1) r1.add(digit, h[1]);
    };
    auto take16 = [&](const uint4 &q) {
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (DT == 0) {
#pragma unroll
                for (int b = 0; b < 4; ++b) take((w[e] >> (8 * b)) & 0xffu);
            } else if (DT == 1) {
                take(w[e] & 0xffffu);
                take(w[e] >> 16);
            } else {
                take(key_f32(__uint_as_float(w[e])));
            }
        }
    };
    if (vec_ok && W % VEC == 0) {
        // this thread's 16-byte chunks, row after row, with the loads of the
        // next two chunks in flight while one is counted
        const int xs = threadIdx.x * VEC, step = blockDim.x * VEC;
        int y = y0, x = xs;
        auto next = [&](int &yy, int &xx) {
            xx += step;
            if (xx >= W) {
                xx = xs;
                yy += ystep;
            }
        };
        auto fetch = [&](int yy, int xx) {
            return __ldg(reinterpret_cast<const uint4 *>(img + (long long)yy * pitch +
                                                        (long long)xx * ES));
        };
        if (xs < W) {
            int y1 = y, x1 = x;
            next(y1, x1);
            uint4 q0 = make_uint4(0, 0, 0, 0), q1 = make_uint4(0, 0, 0, 0);
            if (y < H) q0 = fetch(y, x);
            if (y1 < H) q1 = fetch(y1, x1);
            while (y < H) {
                int y2 = y1, x2 = x1;
                next(y2, x2);
                uint4 q2 = make_uint4(0, 0, 0, 0);
                if (y2 < H) q2 = fetch(y2, x2);
                take16(q0);
                q0 = q1;
                q1 = q2;
                y = y1;
                x = x1;
                y1 = y2;
                x1 = x2;
            }
        }
    } else {
        for (int y = y0; y < H; y += ystep) {
            const char *row = img + (long long)y * pitch;
            for (int x0 = threadIdx.x * VEC; x0 < W; x0 += blockDim.x * VEC) {
                if (vec_ok && x0 + VEC <= W) {
                    take16(__ldg(reinterpret_cast<const uint4 *>(row + (long long)x0 * ES)));
                } else {
                    for (int x = x0; x < x0 + VEC && x < W; ++x) take(load_key<DT>(row, x));
                }
            }
        }
    }
    r0.flush(h[0]);
    r1.flush(h[1]);
}

template <int DT, int BITS>
__device__ __forceinline__ void hist_rows(const char *img, int H, int W, long long pitch,
                                          int pass, const SelState *sel, int y0, int ystep,
                                          HistSmem *hs) {
    if (pass == 0)
        hist_rows_p<DT, BITS, true>(img, H, W, pitch, pass, sel, y0, ystep, hs);
    else
        hist_rows_p<DT, BITS, false>(img, H, W, pitch, pass, sel, y0, ystep, hs);
}

__device__ __forceinline__ void hist_clear(HistSmem *hs) {
    for (int i = threadIdx.x; i < 2 * kRep * kRow; i += blockDim.x) (&hs->v[0][0][0])[i] = 0;
    __syncthreads();
}

__device__ __forceinline__ void hist_flush(HistSmem *hs, SelState *sel) {
    __syncthreads();
    for (int i = threadIdx.x; i < 512; i += blockDim.x) {
        const int g = i >> 8, d = i & 255;
        unsigned v = 0;
#pragma unroll
        for (int r = 0; r < kRep; ++r) v += hs->v[g][r][d];
        if (v) atomicAdd(&sel->hist[g][d], v);
    }
}

template <int DT, int BITS>
__global__ void __launch_bounds__(256) sel_hist(const char *img, int H, int W, long long pitch,
                                                int pass, SelState *sel) {
    __shared__ HistSmem hs;
    hist_clear(&hs);
    hist_rows<DT, BITS>(img, H, W, pitch, pass, sel, blockIdx.x, gridDim.x, &hs);
    hist_flush(&hs, sel);
}

// Pick the digit holding each target's remaining rank; after the last pass
// turn the two keys into the stretch parameters.
template <int DT, int BITS>
__device__ __forceinline__ void pick_digit(int pass, SelState *sel, MhfdStretch *st) {
    __shared__ unsigned cum[2][256];
    __shared__ unsigned pick[2];
    const int t = threadIdx.x;  // 256 threads
    const bool first = (pass == 0);
    for (int g = 0; g < 2; ++g) cum[g][t] = sel->hist[first ? 0 : g][t];
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {  // inclusive scan (Hillis-Steele)
        unsigned a0 = 0, a1 = 0;
        if (t >= o) {
            a0 = cum[0][t - o];
            a1 = cum[1][t - o];
        }
        __syncthreads();
        cum[0][t] += a0;
        cum[1][t] += a1;
        __syncthreads();
    }
    for (int g = 0; g < 2; ++g) {
        const unsigned long long r = sel->rank[g];
        const unsigned long long below = t ? cum[g][t - 1] : 0ull;
        if (r >= below && r < (unsigned long long)cum[g][t]) pick[g] = (unsigned)t;
    }
    __syncthreads();
    if (t < 2) {
        const unsigned d = pick[t];
        const unsigned long long below = d ? cum[t][d - 1] : 0ull;
        sel->rank[t] -= below;
        sel->prefix[t] = (sel->prefix[t] << 8) | d;
    }
    __syncthreads();
    sel->hist[0][t] = 0;
    sel->hist[1][t] = 0;
    if (t == 0 && 8 * (pass + 1) == BITS) {
        const unsigned klo = sel->prefix[0], khi = sel->prefix[1];
        MhfdStretch s;
        if (DT == 2) {
            s.lo = unkey_f32(klo);
            s.hi = unkey_f32(khi);
            s.lo_i = s.hi_i = 0;
        } else {
            s.lo_i = (int)klo;
            s.hi_i = (int)khi;
            s.lo = (float)klo;
            s.hi = (float)khi;
        }
        s.constant = (s.hi == s.lo) ? 1 : 0;
        s.inv = s.constant ? 0.0f : 1.0f / (s.hi - s.lo);
        s.off = s.constant ? 0.0f : -0.5f;
        s.pad = 0;
        *st = s;
    }
}

template <int DT, int BITS>
__global__ void sel_pick(int pass, SelState *sel, MhfdStretch *st) {
    pick_digit<DT, BITS>(pass, sel, st);
}

// ------------------------------------------------------------ batched select
// One launch per pass covers every image of a batch (blockIdx.y = image);
// images whose key width needs fewer passes than the pass index skip.

__device__ __forceinline__ int passes_of(int dtype) { return dtype == 0 ? 1 : (dtype == 1 ? 2 : 4); }

__global__ void bsel_init(const MhfdJob *jobs, SelState *sels, const long long *ranks) {
    const int j = blockIdx.x;
    SelState *sel = sels + j;
    if (threadIdx.x == 0) {
        const unsigned long long n = (unsigned long long)jobs[j].H * (unsigned long long)jobs[j].W;
        sel->prefix[0] = sel->prefix[1] = 0;
        sel->rank[0] = (unsigned long long)ranks[j];
        sel->rank[1] = n - 1 - (unsigned long long)ranks[j];
    }
    for (int i = threadIdx.x; i < 512; i += blockDim.x) (&sel->hist[0][0])[i] = 0;
}

__global__ void __launch_bounds__(256) bsel_hist(const MhfdJob *jobs, SelState *sels, int pass) {
    __shared__ HistSmem hs;
    const MhfdJob job = jobs[blockIdx.y];
    if (pass >= passes_of(job.dtype) || (int)blockIdx.x >= job.H) return;
    hist_clear(&hs);
    SelState *sel = sels + blockIdx.y;
    const char *img = reinterpret_cast<const char *>(job.img);
    if (job.dtype == 0)
        hist_rows<0, 8>(img, job.H, job.W, job.pitch, pass, sel, blockIdx.x, gridDim.x, &hs);
    else if (job.dtype == 1)
        hist_rows<1, 16>(img, job.H, job.W, job.pitch, pass, sel, blockIdx.x, gridDim.x, &hs);
    else
        hist_rows<2, 32>(img, job.H, job.W, job.pitch, pass, sel, blockIdx.x, gridDim.x, &hs);
    hist_flush(&hs, sel);
}

__global__ void bsel_pick(const MhfdJob *jobs, SelState *sels, MhfdStretch *sts, int pass) {
    const MhfdJob job = jobs[blockIdx.x];
    if (pass >= passes_of(job.dtype)) return;
    if (job.dtype == 0)
        pick_digit<0, 8>(pass, sels + blockIdx.x, sts + blockIdx.x);
    else if (job.dtype == 1)
        pick_digit<1, 16>(pass, sels + blockIdx.x, sts + blockIdx.x);
    else
        pick_digit<2, 32>(pass, sels + blockIdx.x, sts + blockIdx.x);
}

template <int DT, int BITS>
int run_select(const void *img, int H, int W, long long pitch, SelState *sel, MhfdStretch *st,
               cudaStream_t s) {
    int dev = 0, sms = 0;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int grid = H < sms * 8 ? H : sms * 8;
    if (grid < 1) grid = 1;
    for (int pass = 0; pass < BITS / 8; ++pass) {
        sel_hist<DT, BITS><<<grid, 256, 0, s>>>(reinterpret_cast<const char *>(img), H, W, pitch,
                                               pass, sel);
        sel_pick<DT, BITS><<<1, 256, 0, s>>>(pass, sel, st);
    }
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

}  // namespace

int enqueue_stretch_batch(const MhfdJob *d_jobs, int n_jobs, int max_passes, int max_rows,
                          const long long *d_ranks, SelState *d_sels, MhfdStretch *d_sts,
                          cudaStream_t s) {
    int dev = 0, sms = 0;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    bsel_init<<<n_jobs, 256, 0, s>>>(d_jobs, d_sels, d_ranks);
    // enough blocks per image to fill the GPU when all images are busy
    int per = (sms * 8 + n_jobs - 1) / n_jobs;
    if (per < 4) per = 4;
    if (per > max_rows) per = max_rows;
    for (int pass = 0; pass < max_passes; ++pass) {
        bsel_hist<<<dim3(per, n_jobs), 256, 0, s>>>(d_jobs, d_sels, pass);
        bsel_pick<<<n_jobs, 256, 0, s>>>(d_jobs, d_sels, d_sts, pass);
    }
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int enqueue_stretch(const void *img, int dtype, int H, int W, long long pitch, long long k,
                    SelState *sel, MhfdStretch *st, cudaStream_t s) {
    const unsigned long long n = (unsigned long long)H * (unsigned long long)W;
    sel_init<<<1, 256, 0, s>>>(sel, (unsigned long long)k, n);
    MHFD_CUDA(cudaGetLastError());
    if (dtype == MHFD_U8) return run_select<0, 8>(img, H, W, pitch, sel, st, s);
    if (dtype == MHFD_U16) return run_select<1, 16>(img, H, W, pitch, sel, st, s);
    return run_select<2, 32>(img, H, W, pitch, sel, st, s);
}

}  // namespace mhfd
