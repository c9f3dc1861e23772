// Device-visible records shared by the library's kernels and by the fused
// detection kernel, which is compiled at run time with NVRTC for each ladder
// (this header is embedded verbatim in that kernel's source).  Plain C
// layout only: no CUDA or host headers.
#ifndef MHFD_TYPES_H
#define MHFD_TYPES_H

// Histogram-stretch bounds of one image (§3), written on the device by the
// order-statistic select kernels and read by the detection kernels.
struct MhfdStretch {
    float lo, hi;    // k-th and (N-1-k)-th smallest values, input units
    float inv;       // 1 / (hi - lo) rounded to f32; 0 for a constant image
    float off;       // -0.5 (centres I' on 0; exact for the DoG), 0 if constant
    int lo_i, hi_i;  // the same bounds as integers (uint8 / uint16 inputs)
    int constant;    // hi == lo
    int pad;
};

// One scale-space maximum: pixel, 0-based DoG layer, response.
struct MhfdCand {
    int x, y, i;
    float resp;
};

// One image of a batch: where it is, how it is stored, where its stretch
// bounds live, which global tile slots and which queue items it owns.
struct MhfdJob {
    const void *img;
    const MhfdStretch *st;
    long long pitch;
    int H, W, dtype, tiles_x, tiles_y;
    int n_tiles;      // tiles of this image (tiles_x * tiles_y)
    int tile_base;    // first global tile slot of this image
    int chunk_base;   // first queue item (chunk of tiles) of this image
    int pad;
};

// By-value parameter block of the fused kernel (the ladder itself is
// compiled into the kernel).  Single image: jobs == nullptr and block b of
// the grid processes the b-th equal share of the image's tiles in
// strip-major order.  Batch: a persistent grid pulls items (chunks of
// `chunk` tiles) from *queue until total_items; item -> (job, tiles)
// through chunk_base.
struct MhfdKHeader {
    const void *img;          // device image, `pitch` bytes per row
    const MhfdStretch *st;    // stretch bounds of this image
    MhfdCand *stage;          // per-tile candidate slots, cap_tile each
    int *tile_count;          // per-tile true candidate count
    float *stack_out;         // optional D output, n planes of H*W
    float *m_out;             // optional max-over-scales output (H*W)
    int *arg_out;             // optional first-argmax output (H*W)
    long long pitch;          // bytes between rows of img
    long long plane;          // H*W (stack plane stride)
    int H, W, dtype, tiles_x, tiles_y, cap_tile;
    float thr;                // feature threshold (strict >)
    const MhfdJob *jobs;      // batch mode: job table (device)
    int *queue;               // batch mode: next item counter (zeroed per launch)
    int n_jobs, total_items;  // batch mode: jobs, queue items (chunks)
    int chunk;                // batch mode: tiles per queue item
    float soft_tau;           // soft-score forward: threshold of the sigmoid
    float soft_inv_t;         //   and its inverse temperature
    int gate;                 // 0 always run; 1 only for an image whose
                              // stretch range is narrow (uint8, or uint16 with
                              // hi - lo <= 4095: the range the tensor-core
                              // vertical pass holds exactly in fp16); 2 only
                              // for the others (per image in a batch)
    double *soft_part;        //   per-block, per-layer sums (zeroed before launch)
    int *flag;                // set to 1 when a bounded wait gives up (or null)
    const void *t2tab;        // two-pass kernel: every level's banded tap
                              // matrices, as its shared-memory buffer holds them
    float *l26val;            // two-pass kernel, 26-neighbour rule: per block,
                              // the responses of kept items ([layer][column][thread])
};

#endif  // MHFD_TYPES_H
