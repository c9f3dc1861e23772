// C ABI of the detector (include/mhfd.h): parameter validation, the ladder
// and taps (§2.2), device scratch, and the asynchronous pipeline
//   stretch select (§3) -> fused detection kernel (§2.2, Eq. 2, Eq. 3)
//   -> tile-ordered gather -> overlap prune -> compaction into pinned memory.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace mhfd {

thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }

int fail(int code, const std::string &msg) {
    t_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    const int code = (e == cudaErrorMemoryAllocation) ? MHFD_ERR_OOM : MHFD_ERR_CUDA;
    return fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace mhfd

using namespace mhfd;

struct mhfd_detector {
    mhfd_params p{};
    int device = 0;
    int n = 0;                   // DoG layers
    std::vector<double> t;       // n+1 Gaussian scales
    std::vector<int> R;          // their radii
    std::vector<float> taps;     // level l: g_l[0..R_l] at tapoff[l]
    std::vector<int> tapoff;
    std::vector<float> tsc;      // t_l as f32 (DoG factor)
    std::vector<double> radius;  // blob radius per DoG layer, sqrt(2) t_i
    double radius_max = 0.0;
    TileConfig cfg;              // FFMA kernel (the tile grid both kernels share)
    LadderKey lk;
    Variant *var = nullptr;
    Variant *var_store = nullptr;
    // tensor-core vertical pass (params.tensor_cores): same tile grid as cfg;
    // takes uint8 and narrow-range uint16 images, the FFMA kernel the rest
    bool use_tc = false;
    TileConfig cfg_tc;
    Variant *var_tc = nullptr;
    Variant *var_tc_store = nullptr;
    Variant *var_soft = nullptr;  // soft-score forward (kernel mode 2)
    // soft-score adjoint: one single-level blur kernel (mode 3) per level
    std::vector<Variant *> var_level;
    std::vector<TileConfig> level_cfg;
    float *soft_D = nullptr;      // the n D planes of the adjoint's forward
    size_t soft_D_px = 0;
    std::vector<uint64_t> params;  // by-value parameter block of the fused kernel
    std::vector<uint64_t> params2; // that of the second (gated) batch launch

    // fixed device buffers
    SelState *sel = nullptr;
    MhfdStretch *st = nullptr;
    Counters *cnt = nullptr;
    double *d_radius = nullptr;
    float *d_sigma = nullptr, *d_radius_f = nullptr, *d_taps = nullptr, *d_tsc = nullptr;
    int *block_tmp = nullptr;
    double *block_sum = nullptr;
    double *soft_part = nullptr;   // per-block layer sums of the soft score
    long long cap = 0;           // candidate list capacity
    MhfdCand *cand = nullptr;
    // two-pass kernel, 26-neighbour rule: per resident block, the responses
    // of the tile's kept items ([layer][128 x strip width])
    float *l26val = nullptr;
    size_t l26val_n = 0;
    // grown with the image
    int cap_tile = 0;
    size_t tiles_cap = 0;
    int *tile_count = nullptr, *tile_off = nullptr;
    MhfdCand *stage = nullptr;
    size_t stage_cap = 0;        // entries
    PruneBuffers pb;
    ConflictTable ct;
    // plain path scratch
    size_t plain_px = 0;
    float *pI = nullptr, *pT = nullptr, *pL = nullptr, *pM = nullptr, *pD = nullptr;
    int *pA = nullptr;
    // host end-to-end copy of the image
    void *d_img_copy = nullptr;
    size_t img_copy_bytes = 0;
    // pinned, device-mapped results
    HostResult *h_res = nullptr, *h_res_dev = nullptr;
    mhfd_blob *h_blobs = nullptr, *h_blobs_dev = nullptr;
    mhfd_blob *h_cands = nullptr, *h_cands_dev = nullptr;
    // device-side result lists, copied (count-exact) at result_wait
    mhfd_blob *d_blobs = nullptr, *d_cands = nullptr;
    bool copied = false;
    cudaEvent_t ev_done = nullptr, ev_t0 = nullptr, ev_k0 = nullptr, ev_k1 = nullptr,
                ev_end = nullptr;
    // batches of images (mhfd_detect_batch)
    struct Batch {
        int cap = 0;                                   // images the arrays hold
        MhfdJob *h_jobs = nullptr, *d_jobs = nullptr;  // job table (pinned + device)
        long long *h_ranks = nullptr, *d_ranks = nullptr;
        SelState *d_sels = nullptr;
        MhfdStretch *d_sts = nullptr;
        int *d_queue = nullptr;
        HostResult *h_res = nullptr, *h_res_dev = nullptr;
        unsigned long long *d_arena_n = nullptr;
        mhfd_blob *d_arena = nullptr;
        unsigned long long arena_cap = 0;
        mhfd_blob *h_arena = nullptr;
        size_t h_arena_cap = 0;
        std::vector<long long> key;                    // shape of the captured graph
        cudaGraphExec_t exec = nullptr;
        cudaStream_t own = nullptr;                    // capture/replay stream
        cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
        bool graphs = true;
        bool pending = false;
        int n = 0;
        bool copied = false;
    } b;
    bool pending = false;
    bool timed = false;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int elem_size(int dtype) { return dtype == MHFD_U8 ? 1 : (dtype == MHFD_U16 ? 2 : 4); }

int build_ladder(const mhfd_params &p, std::vector<double> *t, std::vector<int> *R) {
    if (p.n < 1 || p.n > 63) return fail(MHFD_ERR_INVALID_ARG, "n must be in [1, 63]");
    if (!(p.truncate > 0.0f) || !std::isfinite(p.truncate))
        return fail(MHFD_ERR_INVALID_ARG, "truncate must be positive");
    t->assign(p.n + 1, 0.0);
    if (p.sigmas) {
        for (int i = 0; i <= p.n; ++i) {
            (*t)[i] = p.sigmas[i];
            if (!(p.sigmas[i] > 0.0) || !std::isfinite(p.sigmas[i]))
                return fail(MHFD_ERR_INVALID_ARG, "sigmas must be positive and finite");
            if (i && !(p.sigmas[i] > p.sigmas[i - 1]))
                return fail(MHFD_ERR_INVALID_ARG, "sigmas must increase");
        }
    } else {
        if (!(p.t_min > 0.0) || !(p.t_max > p.t_min) || !std::isfinite(p.t_max))
            return fail(MHFD_ERR_INVALID_ARG, "need 0 < t_min < t_max");
        // §2.2: dt = (max_t - min_t)/n, t_i = min_t + (i-1) dt, i = 1..n+1
        const double dt = (p.t_max - p.t_min) / (double)p.n;
        for (int i = 1; i <= p.n + 1; ++i) (*t)[i - 1] = p.t_min + (double)(i - 1) * dt;
    }
    R->assign(p.n + 1, 0);
    for (int i = 0; i <= p.n; ++i) {
        const double r = std::ceil((double)p.truncate * (*t)[i]);
        if (r < 1.0 || r > 255.0) return fail(MHFD_ERR_UNSUPPORTED, "kernel radius out of range [1, 255]");
        (*R)[i] = (int)r;
    }
    return MHFD_OK;
}

// §2.2: the sampled Gaussian of variance t^2 on k = -R..R, normalised in
// FP64 and rounded to f32; only the symmetric half g[0..R] is kept.
void make_taps(const std::vector<double> &t, const std::vector<int> &R, std::vector<float> *taps,
               std::vector<int> *tapoff, std::vector<float> *tsc) {
    const int nl = (int)t.size();
    taps->clear();
    tsc->clear();
    tapoff->assign(nl + 1, 0);
    for (int l = 0; l < nl; ++l) {
        const int r = R[l];
        std::vector<double> g(2 * r + 1);
        double sum = 0.0;
        for (int k = -r; k <= r; ++k) {
            g[k + r] = std::exp(-((double)k * (double)k) / (2.0 * t[l] * t[l]));
            sum += g[k + r];
        }
        (*tapoff)[l + 1] = (*tapoff)[l] + r + 1;
        for (int k = 0; k <= r; ++k) taps->push_back((float)(g[k + r] / sum));
        tsc->push_back((float)t[l]);
    }
}

int validate_params(const mhfd_params &p) {
    if (!std::isfinite(p.threshold)) return fail(MHFD_ERR_INVALID_ARG, "threshold must be finite");
    if (!(p.overlap >= 0.0f)) return fail(MHFD_ERR_INVALID_ARG, "overlap must be >= 0");
    if (!(p.clip_frac >= 0.0 && p.clip_frac < 0.5))
        return fail(MHFD_ERR_INVALID_ARG, "clip_frac must be in [0, 0.5)");
    if (p.nms != MHFD_NMS_PAPER && p.nms != MHFD_NMS_LOCAL26)
        return fail(MHFD_ERR_INVALID_ARG, "nms must be MHFD_NMS_PAPER or MHFD_NMS_LOCAL26");
    if (p.max_candidates < 1 || p.max_candidates > (1ll << 30))
        return fail(MHFD_ERR_INVALID_ARG, "max_candidates must be in [1, 2^30]");
    if (p.response != MHFD_RESPONSE_DOG && p.response != MHFD_RESPONSE_LOG)
        return fail(MHFD_ERR_INVALID_ARG, "response must be MHFD_RESPONSE_DOG or MHFD_RESPONSE_LOG");
    if (p.boundary != MHFD_BOUNDARY_REFLECT && p.boundary != MHFD_BOUNDARY_PERIODIC)
        return fail(MHFD_ERR_INVALID_ARG, "boundary must be reflect or periodic");
    if (p.tensor_cores < 0 || p.tensor_cores > 2)
        return fail(MHFD_ERR_INVALID_ARG, "tensor_cores must be 0, 1 or 2");
    return MHFD_OK;
}

template <class T>
int dalloc(T **ptr, size_t count) {
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    if (count == 0) count = 1;
    MHFD_CUDA(cudaMalloc(reinterpret_cast<void **>(ptr), count * sizeof(T)));
    return MHFD_OK;
}

int tiles_of(const mhfd_detector *d, int H, int W, int *tx, int *ty) {
    const int TX = d->cfg.tx2 - 2, TY = d->cfg.ty2 - 2;
    *tx = (W + TX - 1) / TX;
    *ty = (H + TY - 1) / TY;
    return (*tx) * (*ty);
}

// Entries of the per-image buffers a detection of an H x W image needs: tile
// counters, candidate staging slots and prune grid cells.  The fused kernel
// stages cap_tile candidates per tile (about 2 B per image pixel); the plain
// path's 16 x 16 tiles stage more (256 or 1024 per tile) and are sized only
// when that path runs.
void image_needs(const mhfd_detector *d, int H, int W, bool plain, size_t *tiles, size_t *stage,
                 size_t *cells) {
    int tx, ty;
    const size_t n_tiles_fused = (size_t)tiles_of(d, H, W, &tx, &ty);
    size_t need_tiles = n_tiles_fused;
    size_t need_stage = n_tiles_fused * (size_t)d->cap_tile;
    if (plain) {
        const size_t n_tiles_plain = (size_t)((W + 15) / 16) * ((H + 15) / 16);
        const size_t cap_tile_plain = d->p.nms == MHFD_NMS_PAPER ? 256 : 1024;
        if (n_tiles_plain > need_tiles) need_tiles = n_tiles_plain;
        if (n_tiles_plain * cap_tile_plain > need_stage) need_stage = n_tiles_plain * cap_tile_plain;
    }
    const int cs = (int)std::ceil(2.0 * d->radius_max) + 1;
    *tiles = need_tiles;
    *stage = need_stage;
    *cells = (size_t)((W + cs - 1) / cs) * ((H + cs - 1) / cs) + 1;
}

int ensure_image_capacity(mhfd_detector *d, int H, int W, bool plain) {
    size_t need_tiles, need_stage, ncells;
    image_needs(d, H, W, plain, &need_tiles, &need_stage, &ncells);
    int rc;
    if (need_tiles > d->tiles_cap) {
        if ((rc = dalloc(&d->tile_count, need_tiles)) || (rc = dalloc(&d->tile_off, need_tiles))) return rc;
        d->tiles_cap = need_tiles;
    }
    if (need_stage > d->stage_cap) {
        if ((rc = dalloc(&d->stage, need_stage))) return rc;
        d->stage_cap = need_stage;
    }
    if (ncells > d->pb.ncells_cap) {
        if ((rc = dalloc(&d->pb.cell_cnt, ncells)) || (rc = dalloc(&d->pb.cell_start, ncells)))
            return rc;
        d->pb.ncells_cap = ncells;
    }
    if (plain) {
        const size_t px = (size_t)H * W;
        if (px > d->plain_px) {
            const size_t nl = d->R.size();
            if ((rc = dalloc(&d->pI, px)) || (rc = dalloc(&d->pT, px)) ||
                (rc = dalloc(&d->pL, px * nl)) || (rc = dalloc(&d->pM, px)) ||
                (rc = dalloc(&d->pA, px)) ||
                (rc = dalloc(&d->pD, d->p.nms == MHFD_NMS_LOCAL26 ? px * (nl - 1) : 1)))
                return rc;
            d->plain_px = px;
        }
    }
    return MHFD_OK;
}

int check_image(const void *img, int dtype, int H, int W, size_t pitch) {
    if (!img) return fail(MHFD_ERR_INVALID_ARG, "image pointer is NULL");
    if (dtype != MHFD_U8 && dtype != MHFD_U16 && dtype != MHFD_F32)
        return fail(MHFD_ERR_INVALID_ARG, "dtype must be MHFD_U8, MHFD_U16 or MHFD_F32");
    if (H < 1 || W < 1) return fail(MHFD_ERR_INVALID_ARG, "H and W must be >= 1");
    if ((long long)H * (long long)W > 2147483647ll) return fail(MHFD_ERR_INVALID_ARG, "H*W must be < 2^31");
    if (pitch < (size_t)W * elem_size(dtype)) return fail(MHFD_ERR_INVALID_ARG, "pitch smaller than a row");
    if (pitch % elem_size(dtype)) return fail(MHFD_ERR_INVALID_ARG, "pitch not a multiple of the element size");
    return MHFD_OK;
}

long long clip_rank(const mhfd_detector *d, int H, int W) {
    const double N = (double)H * (double)W;
    return (long long)std::floor(d->p.clip_frac * N);
}

// fill and launch the fused kernel
int launch_fused(mhfd_detector *d, Variant *v, const void *img, int dtype, int H, int W,
                 size_t pitch, cudaStream_t s, float *d_D, float *d_M, int *d_A, int gate = 0) {
    int tx, ty;
    const int n_tiles = tiles_of(d, H, W, &tx, &ty);
    if ((size_t)v->param_bytes < sizeof(MhfdKHeader) || v->ntaps != (int)d->lk.taps.size())
        return fail(MHFD_ERR_JIT, "kernel parameter layout mismatch");
    d->params.assign((v->param_bytes + 7) / 8 + 1, 0);
    char *pb = reinterpret_cast<char *>(d->params.data());
    MhfdKHeader h;
    std::memset(&h, 0, sizeof(h));
    h.img = img;
    h.st = d->st;
    h.stage = d->stage;
    h.tile_count = d->tile_count;
    h.stack_out = d_D;
    h.m_out = d_M;
    h.arg_out = d_A;
    h.pitch = (long long)pitch;
    h.plane = (long long)H * W;
    h.H = H;
    h.W = W;
    h.dtype = dtype;
    h.tiles_x = tx;
    h.tiles_y = ty;
    h.total_items = n_tiles;
    h.cap_tile = d->cap_tile;
    h.thr = d->p.threshold;
    h.gate = gate;
    h.flag = &d->cnt->ktimeout;
    h.t2tab = v->t2tab;
    h.l26val = d->l26val;
    std::memcpy(pb, &h, sizeof(h));
    void *args[] = {pb};
    // one resident wave: every block marches down an equal share of tiles
    int dev = 0, sms = 1;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long wave = (long long)sms * v->occupancy;
    const unsigned grid = (unsigned)(n_tiles < wave ? n_tiles : wave);
    const CUresult r = drv().launchKernel(v->fn, grid, 1, 1, (unsigned)v->cfg.nt, 1, 1,
                                          (unsigned)v->smem_bytes, (CUstream)s, args, nullptr);
    if (r != CUDA_SUCCESS) {
        const char *es = nullptr;
        drv().getErrorString(r, &es);
        return fail(MHFD_ERR_CUDA, std::string("cuLaunchKernel: ") + (es ? es : "?"));
    }
    return MHFD_OK;
}

int finish_pipeline(mhfd_detector *d, int n_tiles, int cap_tile, int H, int W, cudaStream_t s) {
    int rc = enqueue_gather(d->tile_count, d->stage, n_tiles, cap_tile, d->cap, d->tile_off,
                            d->cand, d->cnt, s);
    if (rc) return rc;
    rc = enqueue_prune(d->cand, d->cnt, d->cap, H, W, d->ct, d->radius_max,
                       (double)d->p.overlap, &d->pb, s);
    if (rc) return rc;
    rc = enqueue_output(d->cand, d->pb.state, d->cnt, d->cap, d->d_sigma, d->d_radius_f, 1,
                        d->h_res_dev, d->d_blobs, d->p.keep_candidates ? d->d_cands : nullptr,
                        d->st, d->block_tmp, d->block_sum, nullptr, 0, s);
    if (rc) return rc;
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_end, s));
    MHFD_CUDA(cudaEventRecord(d->ev_done, s));
    d->pending = true;
    d->copied = false;
    return MHFD_OK;
}

int detect_impl(mhfd_detector *d, const void *img, int dtype, int H, int W, size_t pitch,
                cudaStream_t s, bool store, float *d_D, float *d_M, int *d_A) {
    int rc = check_image(img, dtype, H, W, pitch);
    if (rc) return rc;
    DeviceGuard g(d->device);
    Variant *v = d->var, *vt = d->var_tc;
    if (store) {
        if (!d->var_store) {
            rc = get_variant(d->lk, d->p.nms, 1, d->cfg, &d->var_store);
            if (rc) return rc;
        }
        v = d->var_store;
        if (d->use_tc && !d->var_tc_store) {
            rc = get_variant(d->lk, d->p.nms, 1, d->cfg_tc, &d->var_tc_store);
            if (rc) return rc;
        }
        vt = d->var_tc_store;
    }
    if ((rc = ensure_image_capacity(d, H, W, false))) return rc;
    d->timed = d->p.timing != 0;
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_t0, s));
    rc = enqueue_stretch(img, dtype, H, W, (long long)pitch, clip_rank(d, H, W), d->sel, d->st, s);
    if (rc) return rc;
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_k0, s));
    if (d->use_tc && dtype != MHFD_F32) {
        // uint8 always fits the tensor-core pass; a uint16 image does when
        // its stretch range does (decided on the device: both kernels are
        // launched, gated, and one of them returns at once)
        const bool gated = dtype == MHFD_U16;
        if ((rc = launch_fused(d, vt, img, dtype, H, W, pitch, s, d_D, d_M, d_A, gated ? 1 : 0)))
            return rc;
        if (gated && (rc = launch_fused(d, v, img, dtype, H, W, pitch, s, d_D, d_M, d_A, 2)))
            return rc;
    } else if ((rc = launch_fused(d, v, img, dtype, H, W, pitch, s, d_D, d_M, d_A))) {
        return rc;
    }
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_k1, s));
    int tx, ty;
    const int n_tiles = tiles_of(d, H, W, &tx, &ty);
    return finish_pipeline(d, n_tiles, d->cap_tile, H, W, s);
}

int pinned_alloc(void **h, void **dev, size_t bytes) {
    MHFD_CUDA(cudaHostAlloc(h, bytes ? bytes : 1, cudaHostAllocMapped | cudaHostAllocPortable));
    MHFD_CUDA(cudaHostGetDevicePointer(dev, *h, 0));
    return MHFD_OK;
}

void release(mhfd_detector *d) {
    DeviceGuard g(d->device);
    if (d->pending && d->ev_done) cudaEventSynchronize(d->ev_done);
    void *dev_ptrs[] = {d->sel, d->st, d->cnt, d->d_radius, d->d_sigma, d->d_radius_f, d->d_taps,
                        d->d_tsc, d->block_tmp, d->block_sum, d->cand, d->tile_count,
                        d->tile_off, d->stage, d->pb.cell_cnt, d->pb.cell_start, d->pb.cell_items,
                        d->pb.state, d->pb.nb_idx, d->pb.nb_cnt, d->d_blobs, d->d_cands,
                        d->soft_part, d->pI, d->pT, d->pL, d->pM, d->pD, d->pA, d->d_img_copy,
                        d->soft_D, d->l26val};
    for (void *p : dev_ptrs)
        if (p) cudaFree(p);
    free_conflict_table(&d->ct);
    if (d->b.exec) cudaGraphExecDestroy(d->b.exec);
    if (d->b.own) cudaStreamDestroy(d->b.own);
    if (d->b.ev_fork) cudaEventDestroy(d->b.ev_fork);
    if (d->b.ev_join) cudaEventDestroy(d->b.ev_join);
    void *bdev[] = {d->b.d_jobs, d->b.d_ranks, d->b.d_sels, d->b.d_sts, d->b.d_queue,
                    d->b.d_arena_n, d->b.d_arena};
    for (void *p : bdev)
        if (p) cudaFree(p);
    void *bhost[] = {d->b.h_jobs, d->b.h_ranks, d->b.h_res, d->b.h_arena};
    for (void *p : bhost)
        if (p) cudaFreeHost(p);
    if (d->h_res) cudaFreeHost(d->h_res);
    if (d->h_blobs) cudaFreeHost(d->h_blobs);
    if (d->h_cands) cudaFreeHost(d->h_cands);
    cudaEvent_t evs[] = {d->ev_done, d->ev_t0, d->ev_k0, d->ev_k1, d->ev_end};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    delete d;
}

// The fused kernel's ladder: all n + 1 levels for the DoG; for the LoG
// response the first n levels (one layer each), their second-difference
// taps and t^2 as the layer factors.  *mode gets the tile mode (the rule,
// plus kModeLog for the LoG).
void fused_ladder(const mhfd_params &p, const std::vector<double> &t, const std::vector<int> &R,
                  LadderKey *lk, int *mode) {
    std::vector<int> tapoff;
    std::vector<float> taps, tsc;
    make_taps(t, R, &taps, &tapoff, &tsc);
    lk->boundary = p.boundary;
    lk->response = p.response == MHFD_RESPONSE_LOG ? 1 : 0;
    *mode = p.nms;
    if (!lk->response) {
        lk->R = R;
        lk->taps = taps;
        lk->tsc = tsc;
        lk->taps2.clear();
        return;
    }
    const int n = (int)R.size() - 1;
    *mode = p.nms | kModeLog;
    lk->R.assign(R.begin(), R.begin() + n);
    lk->taps.assign(taps.begin(), taps.begin() + tapoff[n]);
    lk->tsc.clear();
    lk->taps2.clear();
    for (int l = 0; l < n; ++l) {
        lk->tsc.push_back((float)(t[l] * t[l]));
        // g''_k = g_{k-1} - 2 g_k + g_{k+1} of the normalised FP64 taps
        const int r = R[l];
        std::vector<double> g(r + 3, 0.0);
        double sum = 0.0;
        for (int k = -r; k <= r; ++k) sum += std::exp(-((double)k * k) / (2.0 * t[l] * t[l]));
        for (int k = 0; k <= r; ++k) g[k] = std::exp(-((double)k * k) / (2.0 * t[l] * t[l])) / sum;
        auto ge = [&](int k) { return k < 0 ? g[-k] : (k <= r ? g[k] : 0.0); };
        for (int k = 0; k <= r + 1; ++k) lk->taps2.push_back((float)(ge(k - 1) - 2.0 * ge(k) + ge(k + 1)));
    }
}

int resolve_tile(const std::vector<int> &R, int mode, const mhfd_params &p, TileConfig *cfg,
                 bool tc = false) {
    std::string why;
    if (tc && p.tensor_cores == 1 && t2_mode_ok(mode)) {
        // both blur passes on the tensor cores (the default for the paper
        // rule with the DoG response); tile_shape[0] picks the strip width;
        // a ladder too wide for it takes the vertical-pass kernel below
        if (p.tile_shape[0] > 0) {
            *cfg = t2_config((int)R.size(), p.tile_shape[0]);
            if (!t2_shape_ok(R, mode, *cfg, &why))
                return fail(MHFD_ERR_UNSUPPORTED, "tile_shape (two-pass kernel): " + why);
            return MHFD_OK;
        }
        if (choose_tile_t2(R, mode, cfg, &why)) return MHFD_OK;
    }
    if (tc) {
        if (p.tile_shape[0] > 0) {
            const int *ts = p.tile_shape;
            const int nl = (int)R.size();
            if (ts[0] % 4 || ts[0] < 8 || ts[0] > 2048 || ts[1] < 3 || ts[1] > 4096 ||
                ts[4] < 1 || ts[4] > nl)
                return fail(MHFD_ERR_INVALID_ARG, "tile_shape out of range");
            if (ts[5] < 0 || ts[5] > 3 || (ts[5] == 2 && ts[2] % 2))
                return fail(MHFD_ERR_INVALID_ARG, "tile_shape: item kind must be 1, 2 (with an "
                                                  "even number of rows per step) or 3");
            cfg->tx2 = ts[0];
            cfg->ty2 = ts[1];
            cfg->rb = ts[2];
            cfg->nt = ts[3];
            cfg->item = ts[5] == 0 ? 1 : ts[5];
            cfg->gb.assign(ts[4] + 1, 0);
            for (int g = 0; g <= ts[4]; ++g) cfg->gb[g] = (int)((long long)nl * g / ts[4]);
            cfg->tc = 1;
            if (!tc_shape_ok(R, mode, *cfg, &why))
                return fail(MHFD_ERR_UNSUPPORTED, "tile_shape (tensor cores): " + why);
            return MHFD_OK;
        }
        if (p.tile_override > 0) {
            const std::vector<TileConfig> menu = tile_menu_tc(R, mode);
            if (p.tile_override > (int)menu.size())
                return fail(MHFD_ERR_INVALID_ARG, "tile_override out of range");
            *cfg = menu[p.tile_override - 1];
            return MHFD_OK;
        }
        if (!choose_tile_tc(R, mode, cfg, &why)) return fail(MHFD_ERR_UNSUPPORTED, why);
        return MHFD_OK;
    }
    if (p.tile_shape[0] > 0) {
        const int *ts = p.tile_shape;
        const int nl = (int)R.size();
        if (ts[0] % 4 || ts[0] < 8 || ts[0] > 2048 || ts[1] < 3 || ts[1] > 4096 || ts[2] < 2 ||
            ts[2] > 16 || ts[3] % 32 || ts[3] < 32 || ts[3] > 1024 || ts[4] < 1 || ts[4] > nl)
            return fail(MHFD_ERR_INVALID_ARG, "tile_shape out of range");
        if (ts[5] < 0 || ts[5] > 3 || (ts[5] == 2 && ts[2] % 2))
            return fail(MHFD_ERR_INVALID_ARG, "tile_shape: item kind must be 1, 2 (with an "
                                              "even number of rows per step) or 3");
        TileConfig probe;
        probe.tx2 = ts[0];
        probe.rb = ts[2];
        probe.item = ts[5] == 0 ? 1 : ts[5];
        if (h_items(probe) > 2 * ts[3])
            return fail(MHFD_ERR_INVALID_ARG, "tile_shape: more than two horizontal items per thread");
        cfg->tx2 = ts[0];
        cfg->ty2 = ts[1];
        cfg->rb = ts[2];
        cfg->nt = ts[3];
        cfg->item = probe.item;
        cfg->gb.assign(ts[4] + 1, 0);
        for (int g = 0; g <= ts[4]; ++g) cfg->gb[g] = (int)((long long)nl * g / ts[4]);
        if (smem_estimate(R, mode, *cfg) > kSmemLimitBytes)
            return fail(MHFD_ERR_UNSUPPORTED, "tile_shape exceeds shared memory for this ladder");
        return MHFD_OK;
    }
    if (p.tile_override > 0) {
        const std::vector<TileConfig> menu = tile_menu(R, mode);
        if (p.tile_override > (int)menu.size()) return fail(MHFD_ERR_INVALID_ARG, "tile_override out of range");
        *cfg = menu[p.tile_override - 1];
        return MHFD_OK;
    }
    if (!choose_tile(R, mode, cfg, &why)) return fail(MHFD_ERR_UNSUPPORTED, why);
    return MHFD_OK;
}


// ------------------------------------------------------------------ batches

int batch_reserve(mhfd_detector *d, int n, long long total_items, long long total_px,
                  int max_h, int max_w) {
    mhfd_detector::Batch &b = d->b;
    int rc;
    if (n > b.cap) {
        if (b.h_jobs) cudaFreeHost(b.h_jobs);
        if (b.h_ranks) cudaFreeHost(b.h_ranks);
        if (b.h_res) cudaFreeHost(b.h_res);
        b.h_jobs = nullptr;
        b.h_ranks = nullptr;
        b.h_res = nullptr;
        MHFD_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&b.h_jobs), sizeof(MhfdJob) * n, 0));
        MHFD_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&b.h_ranks), sizeof(long long) * n, 0));
        void *hd = nullptr;
        if ((rc = pinned_alloc(reinterpret_cast<void **>(&b.h_res), &hd, sizeof(HostResult) * n)))
            return rc;
        b.h_res_dev = reinterpret_cast<HostResult *>(hd);
        if ((rc = dalloc(&b.d_jobs, n)) || (rc = dalloc(&b.d_ranks, n)) ||
            (rc = dalloc(&b.d_sels, n)) || (rc = dalloc(&b.d_sts, n)))
            return rc;
        b.cap = n;
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        b.key.clear();
    }
    if (!b.d_queue && ((rc = dalloc(&b.d_queue, 2)) || (rc = dalloc(&b.d_arena_n, 1)))) return rc;
    const unsigned long long want = (unsigned long long)(total_px / 32) > (unsigned long long)d->cap
                                        ? (unsigned long long)(total_px / 32)
                                        : (unsigned long long)d->cap;
    if (want > b.arena_cap) {
        if ((rc = dalloc(&b.d_arena, (size_t)want))) return rc;
        b.arena_cap = want;
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        b.key.clear();
    }
    // per-tile slots and counts for every item of the batch
    const size_t items = (size_t)total_items;
    if (items > d->tiles_cap) {
        if ((rc = dalloc(&d->tile_count, items)) || (rc = dalloc(&d->tile_off, items))) return rc;
        d->tiles_cap = items;
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        b.key.clear();
    }
    if (items * (size_t)d->cap_tile > d->stage_cap) {
        if ((rc = dalloc(&d->stage, items * (size_t)d->cap_tile))) return rc;
        d->stage_cap = items * (size_t)d->cap_tile;
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        b.key.clear();
    }
    // the per-image prune grid: capacity for the largest image
    const size_t before = d->pb.ncells_cap;
    if ((rc = ensure_image_capacity(d, max_h, max_w, false))) return rc;
    if (d->pb.ncells_cap != before || d->tiles_cap < items) {
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        b.key.clear();
    }
    return MHFD_OK;
}

// tiles per queue item of a batch: runs of about 256 rows of one strip, long
// enough that the start of a march (the window's first rows, two
// neighbour rows) costs little, short enough to balance the blocks
int batch_chunk(const mhfd_detector *d) {
    const int TY = d->cfg.ty2 - 2;
    const int c = (256 + TY - 1) / TY;
    return c < 1 ? 1 : c;
}

// the whole batch, enqueued on s (also the body of the captured graph)
int batch_enqueue(mhfd_detector *d, int n, int max_passes, int max_rows, long long total_chunks,
                  cudaStream_t s) {
    mhfd_detector::Batch &b = d->b;
    MHFD_CUDA(cudaMemcpyAsync(b.d_jobs, b.h_jobs, sizeof(MhfdJob) * n, cudaMemcpyHostToDevice, s));
    MHFD_CUDA(cudaMemcpyAsync(b.d_ranks, b.h_ranks, sizeof(long long) * n, cudaMemcpyHostToDevice, s));
    MHFD_CUDA(cudaMemsetAsync(b.d_arena_n, 0, sizeof(unsigned long long), s));
    MHFD_CUDA(cudaMemsetAsync(b.d_queue, 0, 2 * sizeof(int), s));
    int rc = enqueue_stretch_batch(b.d_jobs, n, max_passes, max_rows, b.d_ranks, b.d_sels,
                                   b.d_sts, s);
    if (rc) return rc;
    // one persistent launch over every tile of every image; with the
    // tensor-core pass, two gated launches (each takes its images' chunks
    // from its own queue and skips the rest)
    int dev = 0, sms = 1;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_k0, s));
    const int nl = d->use_tc ? 2 : 1;
    for (int k = 0; k < nl; ++k) {
        Variant *v = (d->use_tc && k == 0) ? d->var_tc : d->var;
        std::vector<uint64_t> &pv = k == 0 ? d->params : d->params2;
        pv.assign((v->param_bytes + 7) / 8 + 1, 0);
        MhfdKHeader h;
        std::memset(&h, 0, sizeof(h));
        h.stage = d->stage;
        h.tile_count = d->tile_count;
        h.cap_tile = d->cap_tile;
        h.thr = d->p.threshold;
        h.jobs = b.d_jobs;
        h.queue = b.d_queue + k;
        h.n_jobs = n;
        h.total_items = (int)total_chunks;
        h.chunk = batch_chunk(d);
        h.gate = d->use_tc ? (k == 0 ? 1 : 2) : 0;
        h.flag = &d->cnt->ktimeout;
        h.t2tab = v->t2tab;
        h.l26val = d->l26val;
        std::memcpy(pv.data(), &h, sizeof(h));
        void *args[] = {pv.data()};
        const long long wave = (long long)sms * v->occupancy;
        const unsigned grid = (unsigned)(total_chunks < wave ? total_chunks : wave);
        const CUresult r = drv().launchKernel(v->fn, grid, 1, 1, (unsigned)v->cfg.nt, 1, 1,
                                              (unsigned)v->smem_bytes, (CUstream)s, args, nullptr);
        if (r != CUDA_SUCCESS) return fail(MHFD_ERR_CUDA, "cuLaunchKernel (batch)");
    }
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_k1, s));
    // per image: gather its tiles, prune, compact into the shared blob arena
    for (int j = 0; j < n; ++j) {
        const MhfdJob &jb = b.h_jobs[j];
        rc = enqueue_gather(d->tile_count + jb.tile_base,
                            d->stage + (size_t)jb.tile_base * d->cap_tile, jb.n_tiles,
                            d->cap_tile, d->cap, d->tile_off, d->cand, d->cnt, s);
        if (rc) return rc;
        rc = enqueue_prune(d->cand, d->cnt, d->cap, jb.H, jb.W, d->ct, d->radius_max,
                           (double)d->p.overlap, &d->pb, s);
        if (rc) return rc;
        rc = enqueue_output(d->cand, d->pb.state, d->cnt, d->cap, d->d_sigma, d->d_radius_f, 1,
                            b.h_res_dev + j, b.d_arena, nullptr, b.d_sts + j, d->block_tmp,
                            d->block_sum, b.d_arena_n, b.arena_cap, s);
        if (rc) return rc;
    }
    return MHFD_OK;
}

// The single-level ladder of level l (its radius and taps), compiled as a
// plane blur (kernel mode 3) with its own tile shape.
int level_variant(mhfd_detector *d, int l, Variant **out, TileConfig *cfg) {
    const int nl = (int)d->R.size();
    if ((int)d->var_level.size() != nl) {
        d->var_level.assign(nl, nullptr);
        d->level_cfg.assign(nl, TileConfig());
    }
    if (!d->var_level[l]) {
        LadderKey lk;
        lk.R = {d->R[l]};
        lk.taps.assign(d->taps.begin() + d->tapoff[l], d->taps.begin() + d->tapoff[l] + d->R[l] + 1);
        lk.tsc = {1.0f};
        lk.boundary = d->p.boundary;
        TileConfig c;
        std::string why;
        if (!choose_tile(lk.R, 3, &c, &why)) return fail(MHFD_ERR_UNSUPPORTED, why);
        int rc = get_variant(lk, 3, 0, c, &d->var_level[l]);
        if (rc) return rc;
        d->level_cfg[l] = c;
    }
    *out = d->var_level[l];
    *cfg = d->level_cfg[l];
    return MHFD_OK;
}

// out += B_l in (one level's separable blur of a float32 plane, H x W dense)
int launch_level(mhfd_detector *d, int l, const float *in, float *out, int H, int W,
                 cudaStream_t s) {
    Variant *v;
    TileConfig c;
    int rc = level_variant(d, l, &v, &c);
    if (rc) return rc;
    const int tx = (W + c.tx2 - 3) / (c.tx2 - 2), ty = (H + c.ty2 - 3) / (c.ty2 - 2);
    const long long n_tiles = (long long)tx * ty;
    int dev = 0, sms = 1;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    long long grid = (long long)sms * v->occupancy;
    if (grid > n_tiles) grid = n_tiles;
    std::vector<unsigned long long> pbuf((v->param_bytes + 7) / 8 + 1, 0);
    MhfdKHeader h;
    std::memset(&h, 0, sizeof(h));
    h.img = in;
    h.st = d->st;
    h.pitch = (long long)W * 4;
    h.plane = (long long)H * W;
    h.H = H;
    h.W = W;
    h.dtype = MHFD_F32;
    h.tiles_x = tx;
    h.tiles_y = ty;
    h.total_items = (int)n_tiles;
    h.stack_out = out;
    std::memcpy(pbuf.data(), &h, sizeof(h));
    void *args[] = {pbuf.data()};
    const CUresult r = drv().launchKernel(v->fn, (unsigned)grid, 1, 1, (unsigned)c.nt, 1, 1,
                                          (unsigned)v->smem_bytes, (CUstream)s, args, nullptr);
    if (r != CUDA_SUCCESS) return fail(MHFD_ERR_CUDA, "cuLaunchKernel (level blur)");
    return MHFD_OK;
}

}  // namespace

extern "C" {

void mhfd_default_params(mhfd_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n = 10;
    p->t_min = 1.0;
    p->t_max = 10.0;
    p->sigmas = nullptr;
    p->threshold = 0.1f;
    p->overlap = 0.5f;
    p->nms = MHFD_NMS_PAPER;
    p->truncate = 4.0f;
    p->clip_frac = 0.00175;
    p->max_candidates = 1 << 20;
    p->device = -1;
    p->keep_candidates = 0;
    p->tile_override = 0;
    for (int k = 0; k < 6; ++k) p->tile_shape[k] = 0;
    p->timing = 0;
    p->response = MHFD_RESPONSE_DOG;
    p->boundary = MHFD_BOUNDARY_REFLECT;
    p->tensor_cores = 1;
}

const char *mhfd_last_error(void) { return mhfd::t_err.c_str(); }

const char *mhfd_version(void) { return "mhfd-gb300 0.1 (sm_103a)"; }

int mhfd_create_detector(const mhfd_params *pp, mhfd_detector **out) {
    if (!pp || !out) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    int rc = validate_params(*pp);
    if (rc) return rc;
    mhfd_detector *d = new mhfd_detector();
    d->p = *pp;
    d->p.sigmas = nullptr;  // copied below; the caller's array is not kept
    if ((rc = build_ladder(*pp, &d->t, &d->R))) {
        delete d;
        return rc;
    }
    d->n = pp->n;
    if (pp->device >= 0) {
        d->device = pp->device;
    } else if (cudaGetDevice(&d->device) != cudaSuccess) {
        delete d;
        return fail(MHFD_ERR_CUDA, "no CUDA device");
    }
    DeviceGuard g(d->device);
    const int nl = d->n + 1;
    make_taps(d->t, d->R, &d->taps, &d->tapoff, &d->tsc);
    int tile_mode = d->p.nms;
    fused_ladder(d->p, d->t, d->R, &d->lk, &tile_mode);
    for (int i = 0; i < d->n; ++i) d->radius.push_back(std::sqrt(2.0) * d->t[i]);
    d->radius_max = d->radius[d->n - 1];
    d->use_tc = d->p.tensor_cores != 0 && tc_mode_ok(tile_mode);
    if (d->use_tc) {
        // the tensor-core kernel's shape (tile_shape / tile_override refer to
        // it), and an FFMA companion on the same tile grid
        if ((rc = resolve_tile(d->lk.R, tile_mode, d->p, &d->cfg_tc, true))) {
            delete d;
            return rc;
        }
        if (!companion_tile(d->lk.R, tile_mode, d->cfg_tc, &d->cfg)) {
            delete d;
            return fail(MHFD_ERR_UNSUPPORTED,
                        "no FFMA tile shape shares the tensor-core kernel's strip width");
        }
    } else if ((rc = resolve_tile(d->lk.R, tile_mode, d->p, &d->cfg))) {
        delete d;
        return rc;
    }
    // candidate slots per tile: maxima of the paper rule are at least two
    // pixels apart except on exact plateaus, so 1 per 8 pixels is far above
    // any natural density; a tile beyond it reports MHFD_WARN_OVERFLOW
    const int TXY = (d->cfg.tx2 - 2) * (d->cfg.ty2 - 2);
    d->cap_tile = d->p.nms == MHFD_NMS_PAPER ? (TXY + 7) / 8 : (TXY + 1) / 2;
    d->cap = d->p.max_candidates;
    if ((rc = get_variant(d->lk, d->p.nms, 0, d->cfg, &d->var)) ||
        (d->use_tc && (rc = get_variant(d->lk, d->p.nms, 0, d->cfg_tc, &d->var_tc)))) {
        delete d;
        return rc;
    }
    std::vector<float> sig(64, 0.0f), radf(64, 0.0f);
    std::vector<double> rad(64, 0.0);
    for (int i = 0; i < d->n; ++i) {
        sig[i] = (float)d->t[i];
        radf[i] = (float)d->radius[i];
        rad[i] = d->radius[i];
    }
    if ((rc = dalloc(&d->sel, 1)) || (rc = dalloc(&d->st, 1)) || (rc = dalloc(&d->cnt, 1)) ||
        (rc = dalloc(&d->d_radius, 64)) || (rc = dalloc(&d->d_sigma, 64)) ||
        (rc = dalloc(&d->d_radius_f, 64)) || (rc = dalloc(&d->d_taps, d->taps.size())) ||
        (rc = dalloc(&d->d_tsc, nl)) ||
        (rc = dalloc(&d->block_tmp, 256 + 64)) || (rc = dalloc(&d->block_sum, 256 + 1)) ||
        (rc = dalloc(&d->cand, (size_t)d->cap)) || (rc = dalloc(&d->pb.cell_items, (size_t)d->cap)) ||
        (rc = dalloc(&d->pb.state, (size_t)d->cap)) ||
        (rc = dalloc(&d->pb.nb_idx, (size_t)d->cap * 16)) ||
        (rc = dalloc(&d->pb.nb_cnt, (size_t)d->cap)) ||
        (rc = dalloc(&d->d_blobs, (size_t)d->cap)) ||
        (d->p.keep_candidates && (rc = dalloc(&d->d_cands, (size_t)d->cap)))) {
        release(d);
        return rc;
    }
    if (d->use_tc && d->cfg_tc.tc == 2 && d->p.nms == MHFD_NMS_LOCAL26) {
        int sms = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device) != cudaSuccess) {
            release(d);
            return fail(MHFD_ERR_CUDA, "cudaDeviceGetAttribute failed");
        }
        d->l26val_n = (size_t)sms * d->var_tc->occupancy * (size_t)(nl - 1) * 128 * d->cfg_tc.tx2;
        if ((rc = dalloc(&d->l26val, d->l26val_n))) {
            release(d);
            return rc;
        }
    }
    if (cudaMemset(d->cnt, 0, sizeof(Counters)) ||
        cudaMemcpy(d->d_radius, rad.data(), 64 * sizeof(double), cudaMemcpyHostToDevice) ||
        cudaMemcpy(d->d_sigma, sig.data(), 64 * sizeof(float), cudaMemcpyHostToDevice) ||
        cudaMemcpy(d->d_radius_f, radf.data(), 64 * sizeof(float), cudaMemcpyHostToDevice) ||
        cudaMemcpy(d->d_taps, d->taps.data(), d->taps.size() * sizeof(float), cudaMemcpyHostToDevice) ||
        cudaMemcpy(d->d_tsc, d->tsc.data(), nl * sizeof(float), cudaMemcpyHostToDevice)) {
        release(d);
        return fail(MHFD_ERR_CUDA, "uploading ladder tables failed");
    }
    if (d->p.overlap < 1.0f && (rc = build_conflict_table(d->d_radius, d->radius,
                                                          (double)d->p.overlap, &d->ct))) {
        release(d);
        return rc;
    }
    void *hd = nullptr;
    if ((rc = pinned_alloc(reinterpret_cast<void **>(&d->h_res), &hd, sizeof(HostResult)))) {
        release(d);
        return rc;
    }
    d->h_res_dev = reinterpret_cast<HostResult *>(hd);
    if ((rc = pinned_alloc(reinterpret_cast<void **>(&d->h_blobs), &hd, sizeof(mhfd_blob) * d->cap))) {
        release(d);
        return rc;
    }
    d->h_blobs_dev = reinterpret_cast<mhfd_blob *>(hd);
    if (d->p.keep_candidates) {
        if ((rc = pinned_alloc(reinterpret_cast<void **>(&d->h_cands), &hd, sizeof(mhfd_blob) * d->cap))) {
            release(d);
            return rc;
        }
        d->h_cands_dev = reinterpret_cast<mhfd_blob *>(hd);
    }
    std::memset(d->h_res, 0, sizeof(HostResult));
    if (cudaEventCreateWithFlags(&d->ev_done, cudaEventBlockingSync | cudaEventDisableTiming) ||
        cudaEventCreate(&d->ev_t0) || cudaEventCreate(&d->ev_k0) || cudaEventCreate(&d->ev_k1) ||
        cudaEventCreate(&d->ev_end)) {
        release(d);
        return fail(MHFD_ERR_CUDA, "event creation failed");
    }
    *out = d;
    return MHFD_OK;
}

int mhfd_destroy_detector(mhfd_detector *det) {
    if (!det) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    release(det);
    return MHFD_OK;
}

int mhfd_detect(mhfd_detector *d, const void *img, int32_t dtype, int32_t H, int32_t W,
                size_t pitch, void *stream) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    return detect_impl(d, img, dtype, H, W, pitch, (cudaStream_t)stream, false, nullptr, nullptr,
                       nullptr);
}

int mhfd_debug_stack(mhfd_detector *d, const void *img, int32_t dtype, int32_t H, int32_t W,
                     size_t pitch, void *stream, float *d_D, float *d_M, int32_t *d_arg) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    return detect_impl(d, img, dtype, H, W, pitch, (cudaStream_t)stream, true, d_D, d_M, d_arg);
}

int mhfd_result_wait(mhfd_detector *d, mhfd_result *out) {
    if (!d || !out) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    if (!d->pending) return fail(MHFD_ERR_INVALID_ARG, "no detection enqueued on this detector");
    DeviceGuard g(d->device);
    MHFD_CUDA(cudaEventSynchronize(d->ev_done));
    MHFD_CUDA(cudaGetLastError());
    const HostResult &h = *d->h_res;
    if (!d->copied) {
        const size_t nb = (size_t)(h.c.n_blobs < (unsigned long long)d->cap ? h.c.n_blobs : d->cap);
        if (nb) MHFD_CUDA(cudaMemcpy(d->h_blobs, d->d_blobs, nb * sizeof(mhfd_blob),
                                     cudaMemcpyDeviceToHost));
        if (d->p.keep_candidates && h.c.n_stored)
            MHFD_CUDA(cudaMemcpy(d->h_cands, d->d_cands, (size_t)h.c.n_stored * sizeof(mhfd_blob),
                                 cudaMemcpyDeviceToHost));
        d->copied = true;
    }
    std::memset(out, 0, sizeof(*out));
    out->blobs = d->h_blobs;
    out->n_blobs = (int64_t)h.c.n_blobs;
    out->candidates = d->p.keep_candidates ? d->h_cands : nullptr;
    out->n_candidates = (int64_t)h.c.n_stored;
    out->n_candidates_true = (int64_t)h.c.n_true;
    out->focus_score = (float)h.c.n_blobs;
    out->mean_response = h.c.n_blobs ? (float)(h.sum_resp / (double)h.c.n_blobs) : 0.0f;
    for (int i = 0; i < 64; ++i) out->per_scale[i] = h.per_scale[i];
    out->lo = h.lo;
    out->hi = h.hi;
    if (h.c.timeout & 2) {
        out->status = MHFD_ERR_CHECK;
        return fail(MHFD_ERR_CHECK, "a bounds check of the debug build failed in the fused kernel");
    }
    if (h.c.timeout) {
        out->status = MHFD_ERR_TIMEOUT;
        return fail(MHFD_ERR_TIMEOUT,
                    "a bounded device wait gave up (fused kernel or overlap prune)");
    }
    out->status = h.c.overflow ? MHFD_WARN_OVERFLOW : MHFD_OK;
    return out->status;
}

int mhfd_detect_host_async(mhfd_detector *d, const void *h_img, int32_t dtype, int32_t H,
                           int32_t W, size_t pitch, void *stream) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    int rc = check_image(h_img, dtype, H, W, pitch);
    if (rc) return rc;
    DeviceGuard g(d->device);
    const size_t row = (size_t)W * elem_size(dtype);
    const size_t bytes = row * (size_t)H;
    if (bytes > d->img_copy_bytes) {
        // the previous copy may still be in use by an earlier detection
        if (d->pending && d->ev_done) MHFD_CUDA(cudaEventSynchronize(d->ev_done));
        if ((rc = dalloc(reinterpret_cast<char **>(&d->d_img_copy), bytes))) return rc;
        d->img_copy_bytes = bytes;
    }
    cudaStream_t s = (cudaStream_t)stream;
    MHFD_CUDA(cudaMemcpy2DAsync(d->d_img_copy, row, h_img, pitch, row, (size_t)H,
                                cudaMemcpyHostToDevice, s));
    return detect_impl(d, d->d_img_copy, dtype, H, W, row, s, false, nullptr, nullptr, nullptr);
}

int mhfd_detect_host(mhfd_detector *d, const void *h_img, int32_t dtype, int32_t H, int32_t W,
                     size_t pitch, void *stream, mhfd_result *out) {
    if (!d || !out) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    const int rc = mhfd_detect_host_async(d, h_img, dtype, H, W, pitch, stream);
    if (rc) return rc;
    return mhfd_result_wait(d, out);
}

int mhfd_detect_plain(mhfd_detector *d, const void *img, int32_t dtype, int32_t H, int32_t W,
                      size_t pitch, void *stream) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    int rc = check_image(img, dtype, H, W, pitch);
    if (rc) return rc;
    DeviceGuard g(d->device);
    if ((rc = ensure_image_capacity(d, H, W, true))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    d->timed = d->p.timing != 0;
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_t0, s));
    rc = enqueue_stretch(img, dtype, H, W, (long long)pitch, clip_rank(d, H, W), d->sel, d->st, s);
    if (rc) return rc;
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_k0, s));
    const int cap_tile = d->p.nms == MHFD_NMS_PAPER ? 256 : 1024;
    int n_tiles = 0;
    rc = enqueue_plain(img, dtype, H, W, (long long)pitch, d->st, (int)d->R.size(), d->R,
                       d->d_taps, d->d_tsc, d->p.nms, d->p.threshold, d->pI, d->pT,
                       d->pL, d->pM, d->pA, d->pD, d->tile_count, d->stage, cap_tile,
                       d->p.response, d->p.boundary, &n_tiles, s);
    if (rc) return rc;
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_k1, s));
    return finish_pipeline(d, n_tiles, cap_tile, H, W, s);
}

int mhfd_prune(mhfd_detector *d, const int32_t *x, const int32_t *y, const int32_t *i,
               const float *resp, int64_t n, int32_t H, int32_t W, uint8_t *keep, void *stream) {
    if (!d || !x || !y || !i || !resp || !keep) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n > d->cap) return fail(MHFD_ERR_INVALID_ARG, "n_cand out of [0, max_candidates]");
    if (H < 1 || W < 1) return fail(MHFD_ERR_INVALID_ARG, "H and W must be >= 1");
    DeviceGuard g(d->device);
    int rc = ensure_image_capacity(d, H, W, false);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return MHFD_OK;
    if ((rc = enqueue_pack(x, y, i, resp, n, H, W, d->n, d->cand, d->cnt, s))) return rc;
    if ((rc = enqueue_prune(d->cand, d->cnt, d->cap, H, W, d->ct, d->radius_max,
                            (double)d->p.overlap, &d->pb, s)))
        return rc;
    return enqueue_keep(d->pb.state, d->cnt, n, 1, keep, s);
}

int mhfd_tile_configs(const mhfd_params *p, int32_t *desc, int32_t cap) {
    if (!p) return fail(MHFD_ERR_INVALID_ARG, "NULL params");
    std::vector<double> t;
    std::vector<int> R;
    int rc = build_ladder(*p, &t, &R);
    if (rc) return rc;
    LadderKey lk;
    int mode = p->nms;
    fused_ladder(*p, t, R, &lk, &mode);
    const std::vector<TileConfig> menu =
        p->tensor_cores ? tile_menu_tc(lk.R, mode) : tile_menu(lk.R, mode);
    if (desc) {
        for (int k = 0; k < (int)menu.size() && k < cap; ++k) {
            desc[6 * k + 0] = menu[k].tx2;
            desc[6 * k + 1] = menu[k].ty2;
            desc[6 * k + 2] = menu[k].rb;
            desc[6 * k + 3] = menu[k].nt;
            desc[6 * k + 4] = (int)menu[k].gb.size() - 1;
            desc[6 * k + 5] = menu[k].item;
        }
    }
    return (int)menu.size();
}

int mhfd_chosen_tile(const mhfd_params *p, int32_t *desc6) {
    if (!p || !desc6) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    std::vector<double> t;
    std::vector<int> R;
    int rc = build_ladder(*p, &t, &R);
    if (rc) return rc;
    TileConfig c;
    LadderKey lk;
    int mode = p->nms;
    fused_ladder(*p, t, R, &lk, &mode);
    if ((rc = resolve_tile(lk.R, mode, *p, &c, p->tensor_cores && tc_mode_ok(mode)))) return rc;
    desc6[0] = c.tx2;
    desc6[1] = c.ty2;
    desc6[2] = c.rb;
    desc6[3] = c.nt;
    desc6[4] = (int)c.gb.size() - 1;
    desc6[5] = c.item;
    return MHFD_OK;
}

int mhfd_precompile(const mhfd_params *p, int32_t store) {
    if (!p) return fail(MHFD_ERR_INVALID_ARG, "NULL params");
    int rc = validate_params(*p);
    if (rc) return rc;
    std::vector<double> t;
    std::vector<int> R;
    if ((rc = build_ladder(*p, &t, &R))) return rc;
    LadderKey lk;
    int mode = p->nms;
    fused_ladder(*p, t, R, &lk, &mode);
    std::vector<int> tapoff;
    std::vector<float> taps_all, tsc_all;
    make_taps(t, R, &taps_all, &tapoff, &tsc_all);
    // the shapes a detector with these parameters uses: the tensor-core
    // kernel and its FFMA companion (which the soft score also runs), or the
    // FFMA kernel alone
    TileConfig cfg, ct;
    const bool use_tc = p->tensor_cores && tc_mode_ok(mode);
    if (use_tc) {
        if ((rc = resolve_tile(lk.R, mode, *p, &ct, true))) return rc;
        if (!companion_tile(lk.R, mode, ct, &cfg))
            return fail(MHFD_ERR_UNSUPPORTED,
                        "no FFMA tile shape shares the tensor-core kernel's strip width");
    } else if ((rc = resolve_tile(lk.R, mode, *p, &cfg))) {
        return rc;
    }
    if ((store == 2 || store == 3) && lk.response)
        return fail(MHFD_ERR_UNSUPPORTED, "the soft score uses the DoG response");
    if (store == 2) {  // soft-score forward (its own FFMA shape)
        TileConfig cs;
        std::string why;
        if (!choose_tile(lk.R, 2, &cs, &why)) return fail(MHFD_ERR_UNSUPPORTED, why);
        return precompile_variant(lk, 2, 0, cs);
    }
    if (store == 3) {  // the soft-score adjoint's single-level blurs
        for (size_t l = 0; l < R.size(); ++l) {
            LadderKey l1;
            l1.R = {R[l]};
            l1.taps.assign(taps_all.begin() + tapoff[l], taps_all.begin() + tapoff[l] + R[l] + 1);
            l1.tsc = {1.0f};
            l1.boundary = p->boundary;
            TileConfig c1;
            std::string why;
            if (!choose_tile(l1.R, 3, &c1, &why)) return fail(MHFD_ERR_UNSUPPORTED, why);
            if ((rc = precompile_variant(l1, 3, 0, c1))) return rc;
        }
        return MHFD_OK;
    }
    if (use_tc && (rc = precompile_variant(lk, p->nms, store != 0, ct))) return rc;
    return precompile_variant(lk, p->nms, store != 0, cfg);
}


int mhfd_detect_batch(mhfd_detector *d, int32_t n, const void *const *d_imgs,
                      const int32_t *dtypes, const int32_t *Hs, const int32_t *Ws,
                      const size_t *pitches, void *stream) {
    if (!d || n < 1 || !d_imgs || !dtypes || !Hs || !Ws || !pitches)
        return fail(MHFD_ERR_INVALID_ARG, "NULL argument or n < 1");
    DeviceGuard g(d->device);
    long long total_items = 0, total_px = 0;
    int max_passes = 1, max_h = 1, max_w = 1, max_rows = 1;
    for (int j = 0; j < n; ++j) {
        int rc = check_image(d_imgs[j], dtypes[j], Hs[j], Ws[j], pitches[j]);
        if (rc) return fail(rc, "image " + std::to_string(j) + ": " + mhfd::t_err);
        int tx, ty;
        total_items += tiles_of(d, Hs[j], Ws[j], &tx, &ty);
        total_px += (long long)Hs[j] * Ws[j];
        const int passes = dtypes[j] == MHFD_U8 ? 1 : (dtypes[j] == MHFD_U16 ? 2 : 4);
        max_passes = passes > max_passes ? passes : max_passes;
        max_h = Hs[j] > max_h ? Hs[j] : max_h;
        max_w = Ws[j] > max_w ? Ws[j] : max_w;
    }
    max_rows = max_h;
    if (total_items > 2147483647ll) return fail(MHFD_ERR_INVALID_ARG, "batch too large");
    int rc = batch_reserve(d, n, total_items, total_px, max_h, max_w);
    if (rc) return rc;
    mhfd_detector::Batch &b = d->b;
    std::vector<long long> key;
    key.reserve(4 * n + 2);
    key.push_back(n);
    key.push_back(d->p.timing);
    int base = 0;
    long long chunks = 0;
    const int chunk = batch_chunk(d);
    for (int j = 0; j < n; ++j) {
        int tx, ty;
        const int nt = tiles_of(d, Hs[j], Ws[j], &tx, &ty);
        MhfdJob &jb = b.h_jobs[j];
        std::memset(&jb, 0, sizeof(jb));
        jb.img = d_imgs[j];
        jb.st = b.d_sts + j;
        jb.pitch = (long long)pitches[j];
        jb.H = Hs[j];
        jb.W = Ws[j];
        jb.dtype = dtypes[j];
        jb.tiles_x = tx;
        jb.tiles_y = ty;
        jb.n_tiles = nt;
        jb.tile_base = base;
        jb.chunk_base = (int)chunks;
        base += nt;
        chunks += (nt + chunk - 1) / chunk;
        b.h_ranks[j] = clip_rank(d, Hs[j], Ws[j]);
        key.push_back(Hs[j]);
        key.push_back(Ws[j]);
        key.push_back(dtypes[j]);
        key.push_back((long long)pitches[j]);
    }
    cudaStream_t user = (cudaStream_t)stream;
    d->timed = d->p.timing != 0;
    // the batch runs on a detector-owned stream ordered after the caller's
    // stream and joined back into it (the caller's stream may be the legacy
    // default stream, which cannot be captured)
    if (!b.own) {
        MHFD_CUDA(cudaStreamCreateWithFlags(&b.own, cudaStreamNonBlocking));
        MHFD_CUDA(cudaEventCreateWithFlags(&b.ev_fork, cudaEventDisableTiming));
        MHFD_CUDA(cudaEventCreateWithFlags(&b.ev_join, cudaEventDisableTiming));
    }
    MHFD_CUDA(cudaEventRecord(b.ev_fork, user));
    MHFD_CUDA(cudaStreamWaitEvent(b.own, b.ev_fork, 0));
    cudaStream_t s = b.own;
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_t0, s));
    if (b.graphs && b.exec && key == b.key) {
        MHFD_CUDA(cudaGraphLaunch(b.exec, s));
    } else {
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        b.key.clear();
        bool done = false;
        if (b.graphs && !d->timed) {
            // capture the batch once per shape; later calls with the same
            // shape replay it (the job table travels through pinned memory,
            // so new image pointers need no recapture)
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = batch_enqueue(d, n, max_passes, max_rows, chunks, s);
                e = cudaStreamEndCapture(s, &graph);
                if (rc == MHFD_OK && e == cudaSuccess && graph) {
                    cudaGraphExec_t exec = nullptr;
                    if (cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
                        b.exec = exec;
                        b.key = key;
                        MHFD_CUDA(cudaGraphLaunch(exec, s));
                        done = true;
                    }
                }
                if (graph) cudaGraphDestroy(graph);
            }
            const cudaError_t last = cudaGetLastError();  // refused capture: direct launches
            if (!done) {
                b.graphs = false;
                if (std::getenv("MHFD_DEBUG"))
                    std::fprintf(stderr, "mhfd: batch graph capture refused (rc %d, %s; %s)\n", rc,
                                 cudaGetErrorString(e != cudaSuccess ? e : last),
                                 mhfd::t_err.c_str());
            }
        }
        if (!done && (rc = batch_enqueue(d, n, max_passes, max_rows, chunks, s))) return rc;
    }
    if (d->timed) MHFD_CUDA(cudaEventRecord(d->ev_end, s));
    MHFD_CUDA(cudaEventRecord(d->ev_done, s));
    MHFD_CUDA(cudaEventRecord(b.ev_join, s));
    MHFD_CUDA(cudaStreamWaitEvent(user, b.ev_join, 0));
    b.n = n;
    b.pending = true;
    b.copied = false;
    d->pending = false;
    return MHFD_OK;
}

int mhfd_result_wait_batch(mhfd_detector *d, mhfd_result *outs, int32_t n) {
    if (!d || !outs) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    mhfd_detector::Batch &b = d->b;
    if (!b.pending || n != b.n) return fail(MHFD_ERR_INVALID_ARG, "no batch of this size enqueued");
    DeviceGuard g(d->device);
    MHFD_CUDA(cudaEventSynchronize(d->ev_done));
    MHFD_CUDA(cudaGetLastError());
    unsigned long long used = 0;
    for (int j = 0; j < n; ++j) {
        const unsigned long long e = b.h_res[j].c.blob_base + b.h_res[j].c.n_blobs;
        used = e > used ? e : used;
    }
    if (!b.copied) {
        if (used > b.h_arena_cap) {
            if (b.h_arena) cudaFreeHost(b.h_arena);
            b.h_arena = nullptr;
            MHFD_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&b.h_arena), sizeof(mhfd_blob) * used, 0));
            b.h_arena_cap = used;
        }
        if (used) MHFD_CUDA(cudaMemcpy(b.h_arena, b.d_arena, sizeof(mhfd_blob) * used,
                                       cudaMemcpyDeviceToHost));
        b.copied = true;
    }
    int worst = MHFD_OK;
    for (int j = 0; j < n; ++j) {
        const HostResult &h = b.h_res[j];
        mhfd_result &o = outs[j];
        std::memset(&o, 0, sizeof(o));
        o.blobs = b.h_arena ? b.h_arena + h.c.blob_base : nullptr;
        o.n_blobs = (int64_t)h.c.n_blobs;
        o.candidates = nullptr;
        o.n_candidates = (int64_t)h.c.n_stored;
        o.n_candidates_true = (int64_t)h.c.n_true;
        o.focus_score = (float)h.c.n_blobs;
        o.mean_response = h.c.n_blobs ? (float)(h.sum_resp / (double)h.c.n_blobs) : 0.0f;
        for (int i = 0; i < 64; ++i) o.per_scale[i] = h.per_scale[i];
        o.lo = h.lo;
        o.hi = h.hi;
        o.status = (h.c.timeout & 2) ? MHFD_ERR_CHECK
                   : h.c.timeout     ? MHFD_ERR_TIMEOUT
                                     : (h.c.overflow ? MHFD_WARN_OVERFLOW : MHFD_OK);
        if (o.status == MHFD_ERR_CHECK) worst = MHFD_ERR_CHECK;
        if (o.status == MHFD_ERR_TIMEOUT && worst != MHFD_ERR_CHECK) worst = MHFD_ERR_TIMEOUT;
        else if (o.status == MHFD_WARN_OVERFLOW && worst == MHFD_OK) worst = MHFD_WARN_OVERFLOW;
    }
    if (worst == MHFD_ERR_CHECK)
        return fail(MHFD_ERR_CHECK, "a bounds check of the debug build failed in the fused kernel");
    if (worst == MHFD_ERR_TIMEOUT) return fail(MHFD_ERR_TIMEOUT, "overlap prune did not settle");
    return worst;
}

int mhfd_soft_score(mhfd_detector *d, const void *img, int32_t dtype, int32_t H, int32_t W,
                    size_t pitch, const float *d_w, float tau, float temperature, float grad_s,
                    void *stream, float *d_S, float *d_mean_sig, float *d_dimg, float *d_dw) {
    if (!d || !d_w || !d_S || !d_mean_sig) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    if (!(temperature > 0.0f) || !std::isfinite(tau))
        return fail(MHFD_ERR_INVALID_ARG, "temperature must be > 0 and tau finite");
    if (d->p.response != MHFD_RESPONSE_DOG || d->p.boundary != MHFD_BOUNDARY_REFLECT)
        return fail(MHFD_ERR_UNSUPPORTED,
                    "the soft score uses the DoG response and the reflect boundary");
    int rc = check_image(img, dtype, H, W, pitch);
    if (rc) return rc;
    DeviceGuard g(d->device);
    if ((rc = ensure_image_capacity(d, H, W, d_dimg != nullptr))) return rc;
    constexpr int kMaxBlocks = 2048;
    if (!d->soft_part && (rc = dalloc(&d->soft_part, (size_t)kMaxBlocks * 64))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = enqueue_stretch(img, dtype, H, W, (long long)pitch, clip_rank(d, H, W), d->sel, d->st, s);
    if (rc) return rc;
    if (d_dimg) {
        // forward: the D planes from the stack-storing fused kernel; the
        // per-layer means, S and the level gradients gL_l from them
        const size_t px = (size_t)H * W;
        const int nd = (int)d->R.size() - 1;
        if (px > d->soft_D_px) {
            if ((rc = dalloc(&d->soft_D, px * (size_t)nd))) return rc;
            d->soft_D_px = px;
        }
        if (!d->var_store && (rc = get_variant(d->lk, d->p.nms, 1, d->cfg, &d->var_store)))
            return rc;
        if ((rc = launch_fused(d, d->var_store, img, dtype, H, W, pitch, s, d->soft_D, nullptr,
                               nullptr)))
            return rc;
        if ((rc = enqueue_soft_stack(d->soft_D, (long long)px, nd, d->d_tsc, d_w, tau,
                                     temperature, grad_s, d->soft_part, kMaxBlocks, d_S,
                                     d_mean_sig, d_dw, d->pL, s)))
            return rc;
        // adjoint: the reflect blur is self-adjoint, so gI = sum_l B_l gL_l
        MHFD_CUDA(cudaMemsetAsync(d->pI, 0, sizeof(float) * px, s));
        for (int l = 0; l <= nd; ++l)
            if ((rc = launch_level(d, l, d->pL + (size_t)l * px, d->pI, H, W, s))) return rc;
        return enqueue_soft_mask(img, dtype, H, W, (long long)pitch, d->st, d->pI, d_dimg, s);
    }
    // forward only: the fused kernel accumulates the sigmoids per block
    // (its own FFMA shape: it stores no candidates, so it need not share the
    // detection kernels' tile grid)
    if (!d->var_soft) {
        TileConfig cs;
        std::string why;
        if (!choose_tile(d->lk.R, 2, &cs, &why)) return fail(MHFD_ERR_UNSUPPORTED, why);
        if ((rc = get_variant(d->lk, 2, 0, cs, &d->var_soft))) return rc;
    }
    Variant *v = d->var_soft;
    const int tx = (W + v->cfg.tx2 - 3) / (v->cfg.tx2 - 2), ty = (H + v->cfg.ty2 - 3) / (v->cfg.ty2 - 2);
    const int n_tiles = tx * ty;
    int dev = 0, sms = 1;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    long long grid = (long long)sms * v->occupancy;
    if (grid > n_tiles) grid = n_tiles;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    const int nd = (int)d->R.size() - 1;
    MHFD_CUDA(cudaMemsetAsync(d->soft_part, 0, sizeof(double) * (size_t)grid * nd, s));
    std::vector<unsigned long long> pbuf((v->param_bytes + 7) / 8 + 1, 0);
    MhfdKHeader h;
    std::memset(&h, 0, sizeof(h));
    h.img = img;
    h.st = d->st;
    h.pitch = (long long)pitch;
    h.plane = (long long)H * W;
    h.H = H;
    h.W = W;
    h.dtype = dtype;
    h.tiles_x = tx;
    h.tiles_y = ty;
    h.total_items = n_tiles;
    h.soft_tau = tau;
    h.soft_inv_t = 1.0f / temperature;
    h.soft_part = d->soft_part;
    std::memcpy(pbuf.data(), &h, sizeof(h));
    void *args[] = {pbuf.data()};
    const CUresult r = drv().launchKernel(v->fn, (unsigned)grid, 1, 1, (unsigned)v->cfg.nt, 1, 1,
                                          (unsigned)v->smem_bytes, (CUstream)s, args, nullptr);
    if (r != CUDA_SUCCESS) return fail(MHFD_ERR_CUDA, "cuLaunchKernel (soft forward)");
    return enqueue_soft_finish(d->soft_part, (int)grid, nd, (long long)H * W, d_w, grad_s, d_S,
                               d_mean_sig, d_dw, s);
}

int mhfd_result_ready(mhfd_detector *d) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    if (!d->pending && !d->b.pending) return fail(MHFD_ERR_INVALID_ARG, "nothing enqueued");
    DeviceGuard g(d->device);
    const cudaError_t e = cudaEventQuery(d->ev_done);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return cuda_fail(e, "cudaEventQuery");
}

int mhfd_trim(mhfd_detector *d) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    DeviceGuard g(d->device);
    if (d->ev_done) MHFD_CUDA(cudaEventSynchronize(d->ev_done));
    // a captured batch graph holds the addresses of the buffers freed here
    if (d->b.exec) cudaGraphExecDestroy(d->b.exec);
    d->b.exec = nullptr;
    d->b.key.clear();
    void **grown[] = {reinterpret_cast<void **>(&d->tile_count),
                      reinterpret_cast<void **>(&d->tile_off),
                      reinterpret_cast<void **>(&d->stage),
                      reinterpret_cast<void **>(&d->pb.cell_cnt),
                      reinterpret_cast<void **>(&d->pb.cell_start),
                      reinterpret_cast<void **>(&d->pI), reinterpret_cast<void **>(&d->pT),
                      reinterpret_cast<void **>(&d->pL), reinterpret_cast<void **>(&d->pM),
                      reinterpret_cast<void **>(&d->pD), reinterpret_cast<void **>(&d->pA),
                      reinterpret_cast<void **>(&d->d_img_copy),
                      reinterpret_cast<void **>(&d->soft_D)};
    for (void **p : grown) {
        if (*p) MHFD_CUDA(cudaFree(*p));
        *p = nullptr;
    }
    d->tiles_cap = 0;
    d->stage_cap = 0;
    d->pb.ncells_cap = 0;
    d->plain_px = 0;
    d->img_copy_bytes = 0;
    d->soft_D_px = 0;
    d->pending = false;
    return MHFD_OK;
}

int mhfd_device_bytes(mhfd_detector *d, int32_t H, int32_t W, int64_t *fixed_bytes,
                      int64_t *image_bytes) {
    if (!d || !fixed_bytes || !image_bytes) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    if (H < 0 || W < 0) return fail(MHFD_ERR_INVALID_ARG, "H and W must be >= 0");
    const size_t nl = d->R.size();
    const size_t cap = (size_t)d->cap;
    size_t fixed = sizeof(SelState) + sizeof(MhfdStretch) + sizeof(Counters) +
                   64 * (sizeof(double) + 2 * sizeof(float)) + d->taps.size() * sizeof(float) +
                   nl * sizeof(float) + (256 + 64) * sizeof(int) + (256 + 1) * sizeof(double);
    // candidate list, prune grid items, states, 16 neighbours, counts, blob list
    fixed += cap * (sizeof(MhfdCand) + 3 * sizeof(int) + 16 * sizeof(int) + sizeof(mhfd_blob));
    if (d->p.keep_candidates) fixed += cap * sizeof(mhfd_blob);
    fixed += d->ct.bytes + d->l26val_n * sizeof(float);
    *fixed_bytes = (int64_t)fixed;
    *image_bytes = 0;
    if (H > 0 && W > 0) {
        size_t tiles, stage, cells;
        image_needs(d, H, W, false, &tiles, &stage, &cells);
        *image_bytes = (int64_t)(2 * tiles * sizeof(int) + stage * sizeof(MhfdCand) +
                                 2 * cells * sizeof(int));
    }
    return MHFD_OK;
}

int mhfd_uses_tensor_cores(mhfd_detector *d) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    return d->use_tc ? d->cfg_tc.tc : 0;
}

int mhfd_batch_uses_graph(mhfd_detector *d) {
    if (!d) return fail(MHFD_ERR_INVALID_ARG, "NULL detector");
    return d->b.exec != nullptr ? 1 : 0;
}

int mhfd_last_timing(mhfd_detector *d, float *ms_kernel, float *ms_total) {
    if (!d || !ms_kernel || !ms_total) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    if ((!d->pending && !d->b.pending) || !d->timed)
        return fail(MHFD_ERR_INVALID_ARG, "no timed detection (set params.timing)");
    DeviceGuard g(d->device);
    MHFD_CUDA(cudaEventSynchronize(d->ev_done));
    MHFD_CUDA(cudaEventSynchronize(d->ev_k1));
    MHFD_CUDA(cudaEventSynchronize(d->ev_end));
    MHFD_CUDA(cudaEventElapsedTime(ms_kernel, d->ev_k0, d->ev_k1));
    MHFD_CUDA(cudaEventElapsedTime(ms_total, d->ev_t0, d->ev_end));
    return MHFD_OK;
}

int mhfd_probe_ffma_peak(void *stream, double *ops_per_s) {
    if (!ops_per_s) return fail(MHFD_ERR_INVALID_ARG, "NULL argument");
    return probe_ffma((cudaStream_t)stream, ops_per_s);
}

}  // extern "C"
