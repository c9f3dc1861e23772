// The unfused ("plain") detection pipeline: the comparison baseline of the
// fused kernel and a second, independently written GPU path.
//
// Stretch -> for each Gaussian level a vertical then a horizontal blur
// kernel, each writing a full H x W plane (every L_i lands in device memory,
// as a straightforward per-scale implementation of §2.2 / Algorithm 1 does)
// -> one kernel forming the DoG of Eq. 2 with the running max and first argmax
// over scales (or the whole response stack for the 26-neighbour rule) -> one
// NMS kernel per 16 x 16 tile writing tile-ordered candidates.  Taps and
// radii are read from device memory at run time.
#include "internal.h"

namespace mhfd {

namespace {

constexpr int kT = 16;  // NMS tile edge

// boundary 0: reflect ("d c b a | a b c d | d c b a"); 1: periodic
__device__ __forceinline__ int reflect_i(int i, int n, int boundary = 0) {
    if ((unsigned)i < (unsigned)n) return i;
    if (boundary == 1) {
        int m = i % n;
        return m < 0 ? m + n : m;
    }
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

__global__ void plain_stretch(const char *img, int dtype, int H, int W, long long pitch,
                              const MhfdStretch *stp, float *out) {
    const MhfdStretch st = *stp;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const char *row = img + (long long)y * pitch;
    float f;
    if (dtype == 2) {
        const float v = reinterpret_cast<const float *>(row)[x];
        float u = (v - st.lo) * st.inv;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        f = u + st.off;
    } else {
        int v = dtype == 0 ? (int)reinterpret_cast<const unsigned char *>(row)[x]
                           : (int)reinterpret_cast<const unsigned short *>(row)[x];
        v = min(max(v, st.lo_i), st.hi_i);
        f = fmaf((float)(v - st.lo_i), st.inv, st.off);
    }
    out[(long long)y * W + x] = f;
}

__global__ void plain_vblur(const float *in, int H, int W, const float *taps, int R,
                            float *out, int boundary) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    float acc = 0.0f;
    for (int k = -R; k <= R; ++k)
        acc = fmaf(taps[k < 0 ? -k : k], in[(long long)reflect_i(y + k, H, boundary) * W + x], acc);
    out[(long long)y * W + x] = acc;
}

__global__ void plain_hblur(const float *in, int H, int W, const float *taps, int R,
                            float *out, int boundary) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const float *row = in + (long long)y * W;
    float acc = 0.0f;
    for (int k = -R; k <= R; ++k)
        acc = fmaf(taps[k < 0 ? -k : k], row[reflect_i(x + k, W, boundary)], acc);
    out[(long long)y * W + x] = acc;
}

__global__ void plain_dog(const float *L, long long plane, int n_levels, const float *tsc,
                          int mode, float *M, int *A, float *D) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= plane) return;
    float prev = L[p];
    float m = -__int_as_float(0x7f800000);
    int a = 0;
    for (int l = 1; l < n_levels; ++l) {
        const float cur = L[(long long)l * plane + p];
        const float d = tsc[l - 1] * (cur - prev);
        prev = cur;
        if (mode == 0) {
            if (d > m) {
                m = d;
                a = l - 1;
            }
        } else {
            D[(long long)(l - 1) * plane + p] = d;
        }
    }
    if (mode == 0) {
        M[p] = m;
        A[p] = a;
    }
}

// the scale-normalised Laplacian response t_i^2 grad^2 L_i (5-point stencil,
// neighbours through the blur's boundary), i = 0..n_levels-2, with the same
// max/argmax or stack outputs as plain_dog
__global__ void plain_log(const float *L, int H, int W, int n_levels, const float *tsc, int mode,
                          int boundary, float *M, int *A, float *D) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const long long plane = (long long)H * W;
    const long long p = (long long)y * W + x;
    const int xl = reflect_i(x - 1, W, boundary), xr = reflect_i(x + 1, W, boundary);
    const int yu = reflect_i(y - 1, H, boundary), yd = reflect_i(y + 1, H, boundary);
    float m = -__int_as_float(0x7f800000);
    int a = 0;
    for (int l = 0; l + 1 < n_levels; ++l) {
        const float *Ll = L + (long long)l * plane;
        const float lap = (Ll[(long long)y * W + xl] + Ll[(long long)y * W + xr]) +
                          (Ll[(long long)yu * W + x] + Ll[(long long)yd * W + x]) - 4.0f * Ll[p];
        const float d = tsc[l] * tsc[l] * lap;
        if (mode == 0) {
            if (d > m) {
                m = d;
                a = l;
            }
        } else {
            D[(long long)l * plane + p] = d;
        }
    }
    if (mode == 0) {
        M[p] = m;
        A[p] = a;
    }
}

__device__ __forceinline__ bool is_max8(const float *M, int H, int W, int x, int y, float m) {
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int yy = y + dy, xx = x + dx;
            if ((dx || dy) && yy >= 0 && yy < H && xx >= 0 && xx < W &&
                M[(long long)yy * W + xx] > m)
                return false;
        }
    return true;
}

__device__ __forceinline__ bool is_max26(const float *D, int n, int H, int W, int x, int y, int l,
                                         float v) {
    const long long plane = (long long)H * W;
    for (int dl = -1; dl <= 1; ++dl) {
        const int ll = l + dl;
        if (ll < 0 || ll >= n) continue;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int yy = y + dy, xx = x + dx;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W &&
                    D[ll * plane + (long long)yy * W + xx] > v)
                    return false;
            }
    }
    return true;
}

// one block (kT*kT threads) per tile; ordered compaction in tile raster order
__global__ void __launch_bounds__(kT *kT)
    plain_nms(const float *M, const int *A, const float *D, int n, int H, int W, int mode,
              float thr, int tiles_x, int cap_tile, int *tile_count, MhfdCand *stage) {
    __shared__ int sh_w[kT * kT / 32];
    const int tile = blockIdx.x;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int x = tx * kT + (threadIdx.x % kT), y = ty * kT + (threadIdx.x / kT);
    const bool in = x < W && y < H;
    const long long plane = (long long)H * W;
    int cnt = 0;
    if (in) {
        if (mode == 0) {
            const float m = M[(long long)y * W + x];
            cnt = (m > thr && is_max8(M, H, W, x, y, m)) ? 1 : 0;
        } else {
            for (int l = 0; l < n; ++l) {
                const float v = D[l * plane + (long long)y * W + x];
                if (v > thr && is_max26(D, n, H, W, x, y, l, v)) ++cnt;
            }
        }
    }
    // exclusive scan of counts over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int s = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) sh_w[warp] = s;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kT * kT / 32; ++w) {
        if (w < warp) before += sh_w[w];
        total += sh_w[w];
    }
    int pos = before + s - cnt;
    if (cnt) {
        MhfdCand *dst = stage + (long long)tile * cap_tile;
        if (mode == 0) {
            if (pos < cap_tile) {
                MhfdCand c;
                c.x = x;
                c.y = y;
                c.i = A[(long long)y * W + x];
                c.resp = M[(long long)y * W + x];
                dst[pos] = c;
            }
        } else {
            for (int l = 0; l < n; ++l) {
                const float v = D[l * plane + (long long)y * W + x];
                if (v > thr && is_max26(D, n, H, W, x, y, l, v)) {
                    if (pos < cap_tile) {
                        MhfdCand c;
                        c.x = x;
                        c.y = y;
                        c.i = l;
                        c.resp = v;
                        dst[pos] = c;
                    }
                    ++pos;
                }
            }
        }
    }
    if (threadIdx.x == 0) tile_count[tile] = total;
}

}  // namespace

int enqueue_stack(const void *img, int dtype, int H, int W, long long pitch, const MhfdStretch *st,
                  int n_levels, const std::vector<int> &R, const float *d_taps, float *scratch_I,
                  float *scratch_T, float *scratch_L, cudaStream_t s, int boundary) {
    const dim3 blk(256);
    const dim3 grd((W + 255) / 256, H);
    plain_stretch<<<grd, blk, 0, s>>>(reinterpret_cast<const char *>(img), dtype, H, W, pitch, st,
                                      scratch_I);
    const long long plane = (long long)H * W;
    int off = 0;
    for (int l = 0; l < n_levels; ++l) {
        plain_vblur<<<grd, blk, 0, s>>>(scratch_I, H, W, d_taps + off, R[l], scratch_T, boundary);
        plain_hblur<<<grd, blk, 0, s>>>(scratch_T, H, W, d_taps + off, R[l],
                                        scratch_L + (long long)l * plane, boundary);
        off += R[l] + 1;
    }
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int enqueue_plain(const void *img, int dtype, int H, int W, long long pitch,
                  const MhfdStretch *st, int n_levels, const std::vector<int> &R,
                  const float *d_taps, const float *d_tsc, int mode,
                  float thr, float *scratch_I, float *scratch_T, float *scratch_L,
                  float *scratch_M, int *scratch_A, float *scratch_D, int *tile_count,
                  MhfdCand *stage, int cap_tile, int response, int boundary, int *n_tiles_out,
                  cudaStream_t s) {
    int rc = enqueue_stack(img, dtype, H, W, pitch, st, n_levels, R, d_taps, scratch_I, scratch_T,
                           scratch_L, s, boundary);
    if (rc) return rc;
    const long long plane = (long long)H * W;
    if (response == 1) {
        plain_log<<<dim3((W + 255) / 256, H), 256, 0, s>>>(scratch_L, H, W, n_levels, d_tsc, mode,
                                                           boundary, scratch_M, scratch_A,
                                                           scratch_D);
    } else {
        plain_dog<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(scratch_L, plane, n_levels,
                                                                  d_tsc, mode, scratch_M,
                                                                  scratch_A, scratch_D);
    }
    const int tiles_x = (W + kT - 1) / kT, tiles_y = (H + kT - 1) / kT;
    plain_nms<<<tiles_x * tiles_y, kT * kT, 0, s>>>(scratch_M, scratch_A, scratch_D, n_levels - 1,
                                                   H, W, mode, thr, tiles_x, cap_tile, tile_count,
                                                   stage);
    MHFD_CUDA(cudaGetLastError());
    *n_tiles_out = tiles_x * tiles_y;
    return MHFD_OK;
}

}  // namespace mhfd
