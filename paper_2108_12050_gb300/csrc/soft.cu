// Differentiable soft focus score and its hand-written adjoint.
//
//   S(I, w) = sum_i w_i mean_{x,y} sigmoid((D_i(x,y) - tau) / T)
//
// with D_i the DoG responses of Eq. 2 of the stretched image (stretch bounds
// of §3 held fixed).  The forward alone runs in the fused kernel (mode 2,
// per-block layer sums).  With the backward, the fused kernel's
// stack-storing variant writes the D planes; the kernels here reduce the
// per-layer means in a fixed order (deterministic) and form, for an
// upstream gradient gS, the exact transpose of every linear step:
//   gD_i = gS w_i s_i (1 - s_i) / (T N)                       (elementwise)
//   gL_l = t_{l-1} gD_{l-1} - t_l gD_l                          (DoG adjoint)
//   gI'  = sum_l (H_l V_l)^T gL_l = sum_l H_l V_l gL_l          (blur adjoint)
//   gI   = gI' / (hi - lo) where lo < I < hi, else 0            (clamp mask)
//   gw_i = gS mean_{x,y} s_i
// The blur with symmetric taps and the half-sample symmetric (reflect)
// extension is a symmetric operator, so its adjoint is the blur itself; the
// host runs it as one single-level fused blur kernel (mode 3) per level,
// each adding into gI'.  Nothing is kept between calls.
#include "internal.h"

namespace mhfd {

namespace {

constexpr int kSoftThreads = 256;

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

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

namespace {

// per-block partial sums of the sigmoids of every layer, from the D planes
__global__ void __launch_bounds__(kSoftThreads)
    soft_fwd_d(const float *D, long long plane, int nd, float tau, float inv_t, double *part) {
    __shared__ double sh[kSoftThreads];
    for (int i = 0; i < nd; ++i) {
        double acc = 0.0;
        for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < plane;
             p += (long long)gridDim.x * blockDim.x)
            acc += (double)sigmoidf_((D[(long long)i * plane + p] - tau) * inv_t);
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

// gL_l = t_{l-1} gD_{l-1} - t_l gD_l, l = 0..nd, from the D planes, with
// gD_i = scale w_i s_i (1 - s_i)
__global__ void soft_grad_planes(const float *D, long long plane, int nd, const float *tsc,
                                 const float *w, float tau, float inv_t, float scale,
                                 float *gL) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= plane) return;
    float g_prev = 0.0f, t_prev = 0.0f;
    for (int l = 0; l <= nd; ++l) {
        float g = 0.0f;
        if (l < nd) {
            const float sg = sigmoidf_((D[(long long)l * plane + p] - tau) * inv_t);
            g = scale * w[l] * sg * (1.0f - sg);
        }
        gL[(long long)l * plane + p] = t_prev * g_prev - (l < nd ? tsc[l] * g : 0.0f);
        g_prev = g;
        t_prev = l < nd ? tsc[l] : 0.0f;
    }
}

}  // namespace

int enqueue_soft_stack(const float *d_D, long long plane, int nd, const float *d_tsc,
                       const float *d_w, float tau, float temp, float grad_s, double *block_part,
                       int max_blocks, float *d_S, float *d_mean_sig, float *d_dw, float *d_gL,
                       cudaStream_t s) {
    const float inv_t = 1.0f / temp;
    const long long want = (plane + kSoftThreads - 1) / kSoftThreads;
    const int nb = (int)(want < max_blocks ? want : max_blocks);
    soft_fwd_d<<<nb, kSoftThreads, 0, s>>>(d_D, plane, nd, tau, inv_t, block_part);
    soft_finish<<<1, 64, 0, s>>>(block_part, nb, nd, plane, d_w, grad_s, d_S, d_mean_sig, d_dw);
    const float scale = grad_s * inv_t / (float)plane;
    soft_grad_planes<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(d_D, plane, nd, d_tsc, d_w,
                                                                    tau, inv_t, scale, d_gL);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int enqueue_soft_mask(const void *img, int dtype, int H, int W, long long pitch,
                      const MhfdStretch *st, const float *d_gI, float *d_dimg, cudaStream_t s) {
    const dim3 blk(256), grd((W + 255) / 256, H);
    soft_mask<<<grd, blk, 0, s>>>(reinterpret_cast<const char *>(img), dtype, H, W, pitch, st,
                                  d_gI, d_dimg);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

int enqueue_soft_finish(const double *block_part, int nblocks, int n_layers, long long plane,
                        const float *d_w, float grad_s, float *d_S, float *d_mean_sig, float *d_dw,
                        cudaStream_t s) {
    soft_finish<<<1, 64, 0, s>>>(block_part, nblocks, n_layers, plane, d_w, grad_s, d_S,
                                 d_mean_sig, d_dw);
    MHFD_CUDA(cudaGetLastError());
    return MHFD_OK;
}

}  // namespace mhfd
