// Internal declarations of the detector library (not part of the C ABI).
#ifndef MHFD_INTERNAL_H
#define MHFD_INTERNAL_H

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mhfd.h"
#include "mhfd_types.h"

namespace mhfd {

// ------------------------------------------------------ driver API (lazy)
// The few driver entry points the run-time compiled kernel needs are
// resolved through the runtime (cudaGetDriverEntryPointByVersion), so the
// library itself loads on machines without a GPU driver.
struct DrvApi {
    CUresult (*moduleLoadData)(CUmodule *, const void *);
    CUresult (*moduleUnload)(CUmodule);
    CUresult (*moduleGetFunction)(CUfunction *, CUmodule, const char *);
    CUresult (*moduleGetGlobal)(CUdeviceptr *, size_t *, CUmodule, const char *);
    CUresult (*memcpyDtoH)(void *, CUdeviceptr, size_t);
    CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int);
    CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned,
                             unsigned, unsigned, CUstream, void **, void **);
    CUresult (*getErrorString)(CUresult, const char **);
    CUresult (*occupancy)(int *, CUfunction, int, size_t);
    bool ok;
};
const DrvApi &drv();

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define MHFD_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ------------------------------------------------------- stretch (§3)
// Order-statistic select state (device): one radix-select target per bound.
struct SelState {
    unsigned prefix[2];            // decided high digits of the lo / hi keys
    unsigned long long rank[2];    // remaining rank inside the current prefix
    unsigned hist[2][256];         // digit histograms of the current pass
};

// Enqueue the whole select (init + passes) writing *st.  k = floor(clip*N).
int enqueue_stretch(const void *img, int dtype, int H, int W, long long pitch, long long k,
                    SelState *sel, MhfdStretch *st, cudaStream_t s);

// All images of a batch: one launch per radix pass.  d_ranks[j] = k_j.
int enqueue_stretch_batch(const MhfdJob *d_jobs, int n_jobs, int max_passes, int max_rows,
                          const long long *d_ranks, SelState *d_sels, MhfdStretch *d_sts,
                          cudaStream_t s);

// ---------------------------------------------------- fused kernel (JIT)
// Fused-kernel geometry: strips tx2 - 2 output columns wide, tiles
// (candidate storage units) ty2 - 2 rows high, rb rows per step, nt threads,
// level groups gb.  The input window height follows from these (brows_for).
struct TileConfig {
    int tx2, ty2, rb, nt;
    std::vector<int> gb;   // level-group boundaries
    int tc = 0;            // 1: vertical pass on the tensor cores (tcgen05); 2: both passes
    int item = 1;          // horizontal item: 1 one row x 4 outputs, 2 two rows x 4
                           // (packed FMAs over the row pair), 3 one row x 2 outputs
};
inline int item_rows(const TileConfig &c) { return c.item == 2 ? 2 : 1; }
inline int item_cols(const TileConfig &c) { return c.item == 3 ? 2 : 4; }
// horizontal items of one step of a shape
inline int h_items(const TileConfig &c) { return (c.rb / item_rows(c)) * (c.tx2 / item_cols(c)); }

struct Variant {
    std::string key;
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    int smem_bytes = 0;
    int param_bytes = 0;
    int ntaps = 0;
    int occupancy = 1;  // resident blocks per SM
    TileConfig cfg;
    void *t2tab = nullptr;  // two-pass kernel: its levels' tap matrices (device, built at load)
};

// The ladder as the fused kernel is specialised on: radii, f32 taps (level
// l: g_l[0..R_l] concatenated) and f32 DoG factors t_l.
struct LadderKey {
    std::vector<int> R;
    std::vector<float> taps;
    std::vector<float> tsc;
    int boundary = 0;  // mhfd_boundary of the blur
    int response = 0;  // mhfd_response: 1 = the LoG of each level (taps2: the
                       // second-difference taps g''_l[0..R_l+1] per level)
    std::vector<float> taps2;
};

// Choose a tile configuration for the radii and mode (built-in heuristic).
bool choose_tile(const std::vector<int> &R, int mode, TileConfig *cfg, std::string *why);
// Enumerate the configurations offered to the autotuner.
std::vector<TileConfig> tile_menu(const std::vector<int> &R, int mode);
// opt-in shared memory per block (227 KB) less the kernel's static shared
// variables (the batch loop's queue slot), which count against the same limit
constexpr int kSmemLimitBytes = 232448 - 64;
// added to a kernel mode in the tile and shared-memory helpers: the LoG
// response (one more halo pixel, two V rows per level, a layer per level)
constexpr int kModeLog = 4;
int brows_for(const std::vector<int> &R, int mode, const TileConfig &c);
int smem_estimate(const std::vector<int> &R, int mode, const TileConfig &c);
// Whether the tensor-core vertical pass can take this ladder and mode at all
// (detection rules, DoG response) and whether a shape is valid for it (four
// rows per step, whole warpgroups, tensor-memory columns, shared memory).
bool tc_mode_ok(int mode);
bool tc_shape_ok(const std::vector<int> &R, int mode, const TileConfig &c, std::string *why);
std::vector<TileConfig> tile_menu_tc(const std::vector<int> &R, int mode);
// The two-pass kernel (both blur passes on the tensor cores): its shared
// memory, whether it takes a mode and shape, its configuration for a strip
// width, and the built-in choice.
int t2_smem(const std::vector<int> &R, int mode, const TileConfig &c);
bool t2_mode_ok(int mode);
bool t2_shape_ok(const std::vector<int> &R, int mode, const TileConfig &c, std::string *why);
TileConfig t2_config(int nl, int tx2);
bool choose_tile_t2(const std::vector<int> &R, int mode, TileConfig *cfg, std::string *why);
bool choose_tile_tc(const std::vector<int> &R, int mode, TileConfig *cfg, std::string *why);
// The FFMA kernel's shape on a tensor-core shape's tile grid (the kernel
// that takes the images the tensor-core pass cannot hold exactly).
bool companion_tile(const std::vector<int> &R, int mode, const TileConfig &tc, TileConfig *cfg);
// Compile (or fetch from cache) the fused kernel for this ladder/config.
int get_variant(const LadderKey &lk, int mode, int store, const TileConfig &cfg, Variant **out);
// Compile into the on-disk cache only (no GPU needed).
int precompile_variant(const LadderKey &lk, int mode, int store, const TileConfig &cfg);

// -------------------------------------------------- post-processing kernels
struct Counters {
    unsigned long long n_true;      // candidates found
    unsigned long long n_stored;    // candidates kept in the list
    unsigned long long n_blobs;     // survivors
    int overflow;
    int timeout;
    int ktimeout;                   // bit 0: a fused kernel's bounded wait gave up; bit 1:
                                    // a check of the debug build failed; moved into
                                    // `timeout` (and cleared) by the gather
    unsigned long long blob_base;   // first slot of this image's blobs in the output list
};

struct HostResult {               // mirrored in pinned, device-mapped memory
    Counters c;
    double sum_resp;
    int per_scale[64];
    float lo, hi;
};

struct PruneBuffers {
    int *cell_cnt = nullptr;      // ncells + 1
    int *cell_start = nullptr;    // ncells + 1
    int *cell_items = nullptr;    // cap
    int *state = nullptr;         // cap
    int *nb_idx = nullptr;        // cap * 16 conflicting higher-priority neighbours
    int *nb_cnt = nullptr;        // cap (-1: more than 16, rescan)
    size_t ncells_cap = 0;
};

// Per-detector table of overlap decisions by (scale of kept blob, scale of
// current blob, squared centre distance); see post.cu.
struct ConflictTable {
    int nl = 0;
    const int *lim = nullptr;   // nl*nl: first d2 with zero overlap (0: pair unused)
    const int *off = nullptr;   // nl*nl: word offset of the pair's bitset
    const unsigned *tab = nullptr;
    size_t bytes = 0;           // device bytes of lim, off and tab
};
int build_conflict_table(const double *d_radius, const std::vector<double> &radius,
                         double overlap, ConflictTable *ct);
void free_conflict_table(ConflictTable *ct);

int enqueue_gather(const int *tile_count, const MhfdCand *stage, int n_tiles, int cap_tile,
                   long long cap, int *tile_off, MhfdCand *cand, Counters *cnt,
                   cudaStream_t s);
int enqueue_prune(const MhfdCand *cand, const Counters *cnt, long long cap, int H, int W,
                  const ConflictTable &ct, double radius_max, double overlap, PruneBuffers *pb,
                  cudaStream_t s);
// Compaction of the kept candidates into `blobs`.  With `arena` set, the
// image's slots are reserved at *arena (in stream order) within arena_cap
// entries and the base is published; otherwise they start at 0.
int enqueue_output(const MhfdCand *cand, const int *state, const Counters *cnt, long long cap,
                   const float *d_sigma, const float *d_radius_f, int prune_on,
                   HostResult *h_res_dev, mhfd_blob *blobs, mhfd_blob *h_cands_dev,
                   const MhfdStretch *st, int *block_tmp, double *block_sum,
                   unsigned long long *arena, unsigned long long arena_cap, cudaStream_t s);
// pack caller SoA candidates into the internal list
int enqueue_pack(const int32_t *x, const int32_t *y, const int32_t *i, const float *r,
                 long long n, int H, int W, int n_levels, MhfdCand *cand, Counters *cnt,
                 cudaStream_t s);
int enqueue_keep(const int *state, const Counters *cnt, long long n, int prune_on, uint8_t *keep,
                 cudaStream_t s);

// ------------------------------------------------------------ soft score
// soft score from the D planes (n of them): per-layer means, S, dS/dw and the
// level-gradient planes gL_l (n + 1 of them) of the adjoint
int enqueue_soft_stack(const float *d_D, long long plane, int nd, const float *d_tsc,
                       const float *d_w, float tau, float temp, float grad_s, double *block_part,
                       int max_blocks, float *d_S, float *d_mean_sig, float *d_dw, float *d_gL,
                       cudaStream_t s);
// dimg = gI / (hi - lo) strictly inside (lo, hi), else 0
int enqueue_soft_mask(const void *img, int dtype, int H, int W, long long pitch,
                      const MhfdStretch *st, const float *d_gI, float *d_dimg, cudaStream_t s);
// final reduction of per-block layer sums (fixed order) into S, the
// per-layer means and optionally dS/dw
int enqueue_soft_finish(const double *block_part, int nblocks, int n_layers, long long plane,
                        const float *d_w, float grad_s, float *d_S, float *d_mean_sig, float *d_dw,
                        cudaStream_t s);

// ---------------------------------------------------------- plain path
// I' (stretched, centred) and every Gaussian level L_l as full planes.
int enqueue_stack(const void *img, int dtype, int H, int W, long long pitch, const MhfdStretch *st,
                  int n_levels, const std::vector<int> &R, const float *d_taps, float *scratch_I,
                  float *scratch_T, float *scratch_L, cudaStream_t s, int boundary = 0);
int enqueue_plain(const void *img, int dtype, int H, int W, long long pitch,
                  const MhfdStretch *st, int n_levels, const std::vector<int> &R,
                  const float *d_taps, const float *d_tsc, int mode,
                  float thr, float *scratch_I, float *scratch_T, float *scratch_L,
                  float *scratch_M, int *scratch_A, float *scratch_D, int *tile_count,
                  MhfdCand *stage, int cap_tile, int response, int boundary, int *n_tiles_out,
                  cudaStream_t s);

// ------------------------------------------------------------- probe
int probe_ffma(cudaStream_t s, double *ops_per_s);

}  // namespace mhfd

#endif  // MHFD_INTERNAL_H
