// Differentiable soft focus score and its hand-written adjoint.
//
//   S(I, w) = sum_i w_i mean_{x,y} sigmoid((D_i(x,y) - tau) / T)
//
// with D_i the DoG responses of Eq. 2 of the stretched image (stretch bounds
// of §3 held fixed).  Forward: the Gaussian levels are built as planes (the
// blur kernels of the plain path), then one kernel forms D_i, the sigmoids
// and per-block layer sums, reduced in a fixed order (deterministic).
// Backward, for an upstream gradient gS, by the exact transpose of every
// linear step:
//   gD_i = gS w_i s_i (1 - s_i) / (T N)                       (elementwise)
//   gL_l = t_{l-1} gD_{l-1} - t_l gD_l                          (DoG adjoint)
//   gI'  = sum_l V_l^T H_l^T gL_l                              (blur adjoint)
//   gI   = gI' / (hi - lo) where lo < I < hi, else 0            (clamp mask)
//   gw_i = gS mean_{x,y} s_i
// The blur adjoint gathers, for every output pixel x and tap k, the source
// positions the forward reflect boundary read x from: y + k = x or
// y + k = -1 - x modulo 2n (the mirror), at most one of each family in range.
// The level planes are recomputed for every backward call (nothing is kept
// between forward and backward).
#include "internal.h"

namespace mhfd {

namespace {

constexpr int kSoftThreads = 256;

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// per-block partial sums of the sigmoids of every layer, [block][layer]
__global__ void __launch_bounds__(kSoftThreads)
    soft_fwd(const float *L, long long plane, int nl, const float *tsc, float tau, float inv_t,
             double *part) {
    __shared__ double sh[kSoftThreads];
    const int nd = nl - 1;
    for (int i = 0; i < nd; ++i) {
        double acc = 0.0;
        for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < plane;
             p += (long long)gridDim.x * blockDim.x) {
            const float d = tsc[i] * (L[(long long)(i + 1) * plane + p] - L[(long long)i * plane + p]);
            acc += (double)sigmoidf_((d - tau) * inv_t);
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int o = kSoftThreads / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(long long)blockIdx.x * nd + i] = sh[0];
        __syncthreads();
    }
}

__global__ void soft_finish(const double *part, int nblocks, int nd, long long plane,
                            const float *w, float grad_s, float *S, float *mean_sig, float *dw) {
    __shared__ double ms[64];
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += part[(long long)b * nd + i];
        ms[i] = acc / (double)plane;
        mean_sig[i] = (float)ms[i];
        if (dw) dw[i] = (float)(grad_s * ms[i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nd; ++i) s += (double)w[i] * ms[i];
        *S = (float)s;
    }
}

// gL_l in place of L_l (levels in ascending order: D_l is formed from the
// untouched L_l and L_{l+1} before L_l is overwritten)
__global__ void soft_dog_adjoint(float *L, long long plane, int nl, const float *tsc,
                                 const float *w, float tau, float inv_t, float scale) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= plane) return;
    const int nd = nl - 1;
    float g_prev = 0.0f;  // gD_{l-1}
    float t_prev = 0.0f;
    float l_cur = L[p];
    for (int l = 0; l < nl; ++l) {
        float g = 0.0f;
        float l_next = 0.0f;
        if (l < nd) {
            l_next = L[(long long)(l + 1) * plane + p];
            const float d = tsc[l] * (l_next - l_cur);
            const float sg = sigmoidf_((d - tau) * inv_t);
            g = scale * w[l] * sg * (1.0f - sg);
        }
        const float gl = t_prev * g_prev - (l < nd ? tsc[l] * g : 0.0f);
        L[(long long)l * plane + p] = gl;
        g_prev = g;
        t_prev = l < nd ? tsc[l] : 0.0f;
        l_cur = l_next;
    }
}

__device__ __forceinline__ int mod2n(int v, int n2) {
    int m = v % n2;
    return m < 0 ? m + n2 : m;
}

// transpose of the row pass: out(y, x) = sum_k g_|k| sum_{x' : reflect(x'+k) = x} in(y, x')
__global__ void hblur_adjoint(const float *in, int H, int W, const float *taps, int R, float *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const float *row = in + (long long)y * W;
    const int w2 = 2 * W;
    float acc = 0.0f;
    if (x >= R && x + R < W) {  // away from the borders only the direct term exists
        for (int k = -R; k <= R; ++k) acc = fmaf(taps[k < 0 ? -k : k], row[x - k], acc);
        out[(long long)y * W + x] = acc;
        return;
    }
    for (int k = -R; k <= R; ++k) {
        const float g = taps[k < 0 ? -k : k];
        const int a = mod2n(x - k, w2);
        if (a < W) acc = fmaf(g, row[a], acc);
        const int b = mod2n(-1 - x - k, w2);
        if (b < W) acc = fmaf(g, row[b], acc);
    }
    out[(long long)y * W + x] = acc;
}

// transpose of the column pass, accumulated into out
__global__ void vblur_adjoint_acc(const float *in, int H, int W, const float *taps, int R,
                                  float *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const int h2 = 2 * H;
    float acc = 0.0f;
    if (y >= R && y + R < H) {
        for (int k = -R; k <= R; ++k)
            acc = fmaf(taps[k < 0 ? -k : k], in[(long long)(y - k) * W + x], acc);
        out[(long long)y * W + x] += acc;
        return;
    }
    for (int k = -R; k <= R; ++k) {
        const float g = taps[k < 0 ? -k : k];
        const int a = mod2n(y - k, h2);
        if (a < H) acc = fmaf(g, in[(long long)a * W + x], acc);
        const int b = mod2n(-1 - y - k, h2);
        if (b < H) acc = fmaf(g, in[(long long)b * W + x], acc);
    }
    out[(long long)y * W + x] += acc;
}

// clamp mask and 1/(hi - lo): the stretch passes gradient only strictly
// inside (lo, hi)
__global__ void soft_mask(const char *img, int dtype, int H, int W, long long pitch,
                          const MhfdStretch *stp, const float *gI, float *dimg) {
    const MhfdStretch st = *stp;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const char *row = img + (long long)y * pitch;
    bool inside;
    if (dtype == 2) {
        const float v = reinterpret_cast<const float *>(row)[x];
        inside = v > st.lo && v < st.hi;
    } else {
        const int v = dtype == 0 ? (int)reinterpret_cast<const unsigned char *>(row)[x]
                                 : (int)reinterpret_cast<const unsigned short *>(row)[x];
        inside = v > st.lo_i && v < st.hi_i;
    }
    const long long p = (long long)y * W + x;
    dimg[p] = (inside && !st.constant) ? gI[p] * st.inv : 0.0f;
}

}  // namespace

int enqueue_soft_finish(const double *block_part, int nblocks, int n_layers, long long plane,
                        const float *d_w, float grad_s, float *d_S, float *d_mean_sig, float *d_dw,
                        cudaStream_t s) {
    soft_finish<<<1, 64, 0, s>>>(block_part, nblocks, n_layers, plane, d_w, grad_s, d_S,
                                 d_mean_sig, d_dw);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int enqueue_soft(const void *img, int dtype, int H, int W, long long pitch, const MhfdStretch *st,
                 int n_levels, const std::vector<int> &R, const float *d_taps, const float *d_tsc,
                 const float *d_w, float tau, float temp, float grad_s, float *scratch_L,
                 float *scratch_T, float *scratch_G, double *block_part, int max_blocks,
                 float *d_S, float *d_mean_sig, float *d_dimg, float *d_dw, cudaStream_t s) {
    const long long plane = (long long)H * W;
    int rc = enqueue_stack(img, dtype, H, W, pitch, st, n_levels, R, d_taps, scratch_G, scratch_T,
                           scratch_L, s);
    if (rc) return rc;
    const int nd = n_levels - 1;
    const float inv_t = 1.0f / temp;
    long long want = (plane + kSoftThreads - 1) / kSoftThreads;
    const int nb = (int)(want < max_blocks ? want : max_blocks);
    soft_fwd<<<nb, kSoftThreads, 0, s>>>(scratch_L, plane, n_levels, d_tsc, tau, inv_t, block_part);
    soft_finish<<<1, 64, 0, s>>>(block_part, nb, nd, plane, d_w, grad_s, d_S, d_mean_sig, d_dw);
    MHFD_CUDA(cudaGetLastError());
    if (!d_dimg) return MHFD_OK;
    const float scale = grad_s * inv_t / (float)plane;
    soft_dog_adjoint<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(scratch_L, plane, n_levels,
                                                                    d_tsc, d_w, tau, inv_t, scale);
    // scratch_G (the stretched image, no longer needed) accumulates gI'
    MHFD_CUDA(cudaMemsetAsync(scratch_G, 0, sizeof(float) * plane, s));
    const dim3 blk(256), grd((W + 255) / 256, H);
    int off = 0;
    for (int l = 0; l < n_levels; ++l) {
        hblur_adjoint<<<grd, blk, 0, s>>>(scratch_L + (long long)l * plane, H, W, d_taps + off,
                                          R[l], scratch_T);
        vblur_adjoint_acc<<<grd, blk, 0, s>>>(scratch_T, H, W, d_taps + off, R[l], scratch_G);
        off += R[l] + 1;
    }
    soft_mask<<<grd, blk, 0, s>>>(reinterpret_cast<const char *>(img), dtype, H, W, pitch, st,
                                  scratch_G, d_dimg);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

}  // namespace mhfd
