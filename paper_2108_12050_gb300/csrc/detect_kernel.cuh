// Fused multi-scale feature detection kernel (sm_103a).
//
// Compiled at run time with NVRTC once per ladder: the host prepends MHFD_*
// macros (number of Gaussian levels, their radii, the f32 tap values and
// scale factors as exact hexadecimal literals, tile geometry, mode) so that
// every loop over scales and taps is fully unrolled and every tap is an
// immediate operand of its FFMA (no constant-memory load per multiply).
//
// The image is cut into vertical strips TX pixels wide; a strip into tiles
// of TY rows, the unit of candidate storage.  A CTA marches down a run of
// consecutive tiles of one strip (a "chunk"), RB output rows per step:
//   1. the input rows of the halo'd strip (RMAX+1 pixels of halo, reflect
//      boundary "d c b a | a b c d | d c b a" or periodic, histogram stretch
//      of §3 applied on the fly) live in a sliding shared-memory window of BROWS rows; the
//      RB rows the next step needs are fetched into registers at the start of
//      a step and written after it (their latency hides behind the step), and
//      every few steps the window is shifted back to the buffer's start;
//   2. per step and per group of levels, a vertical pass computes
//      V_l = g_l (*)_y I' for every column of the group's halo'd width: each
//      thread owns a column, forms the folded sums I'(y+k) + I'(y-k) once and
//      feeds them to all levels of the group (taps are symmetric, §2.2), for
//      up to four rows at a time; or (MHFD_VTC, "tensor-core vertical pass"
//      below) the window holds exact fp16 integers and the vertical pass is
//      a product with banded tap matrices on the tensor cores (tcgen05),
//      issued a step ahead and read back from tensor memory;
//   3. a horizontal pass computes L_l = g_l (*)_x V_l for four adjacent
//      outputs per thread from float4 shared-memory reads and forms the DoG
//      of Eq. 2, D_{l-1} = t_{l-1} (L_l - L_{l-1}), in registers;
//   4. the paper's rule (Eq. 3) keeps the running max over scales and its
//      first argmax in registers and compares it with its 3x3 neighbourhood
//      from a (RB+2)-row ring in shared memory; the 26-neighbour mode keeps a
//      ring of the whole response stack instead.  The ring carries over from
//      step to step, so rows are computed once per chunk, not once per tile;
//   5. features above the threshold are compacted in row-major order within
//      each tile (block scan) into that tile's slots of the candidate list.
// The response stack never reaches global memory (except in the STORE
// variant used by the tests).

#ifndef MHFD_NL
#error "MHFD_* configuration macros must be defined before this source"
#endif

namespace mk {

#define MK_HD __host__ __device__

constexpr int NL = MHFD_NL;
// Response: 0 the DoG of Eq. 2 over NL levels (NL - 1 layers); 1 the
// scale-normalised Laplacian t_l^2 grad^2 L_l of each of NL levels (NL
// layers), with the 5-point second differences folded into derived taps:
// dyy L = H (g'' (*)_y I) and dxx L = g'' (*)_x (V I), g''_k = g_{k-1} -
// 2 g_k + g_{k+1} (radius R + 1), so both share the vertical folded sums.
constexpr bool LOG = (MHFD_RESPONSE) == 1;
constexpr int NDOG = LOG ? NL : NL - 1;  // response layers
constexpr int NGROUPS = MHFD_NGROUPS;
constexpr int TX2 = MHFD_TX2;
constexpr int TX = TX2 - 2;       // output columns of a strip
constexpr int TY = MHFD_TY2 - 2;  // output rows of a tile (candidate storage unit)
constexpr int RB = MHFD_RB;
constexpr int NT = MHFD_NT;
// 0: paper rule (argmax over scales + 3x3), 1: 3x3x3 rule, 2: soft-score
// forward (per-layer sums of sigmoid((D - tau) / T), no maxima), 3: blur of
// a float32 plane by the single level of the ladder, added into the output
// plane (no stretch, no maxima; the soft-score adjoint runs one per level)
constexpr int MODE = MHFD_MODE;
constexpr bool STORE = (MHFD_STORE) != 0;
// Vertical pass on the tensor cores (tcgen05, see "tensor-core vertical
// pass" below) instead of FFMA; detection modes, DoG, integer images.
#ifndef MHFD_VTC
#define MHFD_VTC 0
#endif
constexpr bool TC = (MHFD_VTC) == 1;
// Both blur passes on the tensor cores (MHFD_VTC 2, "two-pass kernel" below):
// detection with the DoG response (the paper rule, the 26-neighbour rule up
// to 16 layers), integer images.
constexpr bool TC2 = (MHFD_VTC) == 2;
// Rows per horizontal item: 1 (four outputs of one row), or 2 (four
// outputs of each of two adjacent rows; the V rows of a step are then
// stored pair-interleaved, column by column, so that one float4 load holds
// two columns of both rows and each tap is one packed two-lane FMA over the
// row pair, the same tap in both lanes).  The detection modes only.
#ifndef MHFD_HR
#define MHFD_HR 1
#endif
constexpr int HR = MHFD_HR;
// Outputs per row of a horizontal item: 4 (float4 loads, each value feeding
// four outputs), or 2 (one-row items only: twice the items per step, for
// shapes whose strips are too narrow to give every thread a four-output item)
#ifndef MHFD_HW
#define MHFD_HW 4
#endif
constexpr int HW = MHFD_HW;
// one-row items on packed two-lane FMAs over column pairs (outputs (0, 1)
// and (2, 3)): measured faster for the tensor-core LoG kernel (2.79 -> 2.61
// ms on a 4096^2 tile), slower for the DoG kernels (1.00 -> 1.16 ms
// tensor-core, 1.51 -> 1.60 ms FFMA)
constexpr bool HPACK = TC && LOG && HR == 1 && HW == 4;
// Debug build (MHFD_CHECKS 1): the shared-memory and global indices the
// kernel forms are checked against their buffers; a failed check sets bit 1
// of the kernel's flag word (the host reports MHFD_ERR_CHECK) and the
// access is skipped (a load reads 0) - no trap, the context stays usable.
#ifndef MHFD_CHECKS
#define MHFD_CHECKS 0
#endif
constexpr bool CHECKS = (MHFD_CHECKS) != 0;
__shared__ int *mk_chk_flag;
__device__ __forceinline__ bool mk_ok(bool cond) {
    if constexpr (CHECKS) {
        if (!cond && mk_chk_flag) atomicOr(mk_chk_flag, 2);
        return cond;
    }
    return true;
}

// Kernel radius R_l of Gaussian level l and the level groups [GB(g), GB(g+1)).
MK_HD constexpr int kR(int l) {
    constexpr int r[NL] = {MHFD_RLIST};
    return r[l];
}
MK_HD constexpr int kGB(int g) {
    constexpr int b[NGROUPS + 1] = {MHFD_GB};
    return b[g];
}
// f32 Gaussian taps (level l: g_l[0..R_l] at tapoff(l)) and DoG factors t_l.
// Only ever evaluated in constant expressions (template-constant indices),
// so every tap becomes an immediate operand of its FFMA.
MK_HD constexpr float kTap(int i) {
    constexpr float a[] = {MHFD_TAPS};
    return a[i];
}
MK_HD constexpr float kTsc(int l) {
    constexpr float a[] = {MHFD_TSC};
    return a[l];
}
// LoG: the second-difference taps g''_l[0..R_l+1] at tapoff2(l)
MK_HD constexpr float kTap2(int i) {
    constexpr float a[] = {MHFD_TAPS2};
    return a[i];
}
template <int I>
__device__ __forceinline__ float tap() {
    constexpr float v = kTap(I);
    return v;
}
template <int I>
__device__ __forceinline__ float tap2() {
    constexpr float v = kTap2(I);
    return v;
}
// halo a level needs: its radius, one more for the second-difference taps
MK_HD constexpr int kRH(int l) { return kR(l) + (LOG ? 1 : 0); }
MK_HD constexpr int rmax_of() {
    int m = 0;
    for (int l = 0; l < NL; ++l) m = kRH(l) > m ? kRH(l) : m;
    return m;
}
constexpr int RMAX = rmax_of();
// the largest halo radius among the levels of group g
MK_HD constexpr int group_rmax(int g) {
    int m = 0;
    for (int l = kGB(g); l < kGB(g + 1); ++l) m = kRH(l) > m ? kRH(l) : m;
    return m;
}
constexpr int WEXT = TX2 + 2 * RMAX;           // columns of the halo'd strip
constexpr int WEXTP = (WEXT + 3) & ~3;
constexpr int WIN = RB + 2 * RMAX;             // input rows one step reads
constexpr int BROWS = MHFD_BROWS;              // rows of the sliding input window
constexpr int NT_COLS = (WEXT + MHFD_NT - 1) / MHFD_NT;  // input columns per thread
constexpr int RING = RB + 2;
constexpr int NQW = TX2 / HW;                  // horizontal items per row
constexpr int HITEMS = (RB / HR) * NQW;
// threads that take horizontal items: with the tensor-core pass and a
// block of whole warpgroups plus one warp, that last warp only issues MMAs
constexpr int NTW = (TC && NT % 128 == 32) ? NT - 32 : NT;
constexpr int HI = (HITEMS + NTW - 1) / NTW;
constexpr int NPARTS = (RB + 3) / 4;

// padded width of the V row of level l (its outputs plus its own halo);
// LoG levels hold two rows, V and g'' (*)_y I, side by side
MK_HD constexpr int extp(int l) { return (TX2 + 2 * kRH(l) + 3) & ~3; }
MK_HD constexpr int vwidth(int l) { return LOG ? 2 * extp(l) : extp(l); }
// taps of level l start at tapoff(l) of the parameter block
MK_HD constexpr int tapoff(int l) {
    int o = 0;
    for (int j = 0; j < l; ++j) o += kR(j) + 1;
    return o;
}
MK_HD constexpr int tapoff2(int l) {
    int o = 0;
    for (int j = 0; j < l; ++j) o += kR(j) + 2;
    return o;
}
MK_HD constexpr int group_of(int l) {
    int g = 0;
    while (g + 1 < NGROUPS && kGB(g + 1) <= l) ++g;
    return g;
}
// the V row of level l starts at voff(l) within its group's row
MK_HD constexpr int voff(int l) {
    int o = 0;
    for (int j = kGB(group_of(l)); j < l; ++j) o += vwidth(j);
    return o;
}
MK_HD constexpr int vrow_max() {
    int m = 0;
    for (int g = 0; g < NGROUPS; ++g) {
        int o = 0;
        for (int j = kGB(g); j < kGB(g + 1); ++j) o += vwidth(j);
        m = o > m ? o : m;
    }
    return m;
}
constexpr int NTAPS = tapoff(NL);
constexpr int VROW = vrow_max();
// Shared-memory index of column cc of the V row `part` (1: the LoG's
// second row) of level L at step row j.  One-row items: rows one after
// another.  Two-row items: a row pair holds, per level and part, a float2
// (both rows) per column, the columns ordered by their residue mod 4 -
// column cc at (cc mod 4) * extp(L) / 4 + cc / 4 - so that the loads of
// one window column by the warp's items (columns 4q + M, q = item) are
// contiguous.
MK_HD constexpr int vidx(int L, int part, int j, int cc) {
    return HR == 1 ? j * VROW + voff(L) + part * extp(L) + cc
                   : (j >> 1) * 2 * VROW + 2 * (voff(L) + part * extp(L)) +
                         2 * ((cc & 3) * (extp(L) >> 2) + (cc >> 2)) + (j & 1);
}

// Tensor-core vertical pass geometry.  The window holds the centred integer
// pixels x = clamp(v, lo, hi) - c0 as fp16 (exact while |x| <= 2048) in the
// canonical no-swizzle MN-major operand layout of tcgen05: column group cg
// (8 columns, 16 bytes per row) at cg * TC_GSTR, row r at + 16 r.  M tiles
// of 128 window columns; per level group G a K range of RB + 2 RG window
// rows (padded to 16) and N = (levels of G) x RB accumulator columns (padded
// to 16): one B matrix per group and tap part (hi, lo).
constexpr int TC_NMT = (WEXT + 127) / 128;
constexpr int TC_WT = 128 * TC_NMT;
constexpr int TC_CG = TC_WT / 8;
constexpr int TC_CGL = (WEXT + 7) / 8;  // column groups holding image columns
constexpr int TC_GSTR = ((16 * BROWS + 127) / 128) * 128 + 32;  // 4 groups cover the 32 banks
constexpr int TC_WIN_BYTES = TC ? TC_CG * TC_GSTR : 0;
constexpr float TC_S = 1024.0f;  // tap scale: keeps the lo parts of small taps normal in fp16
constexpr int SMEM_IN = TC ? 0 : BROWS * WEXTP;
constexpr int SMEM_V = RB * VROW;
constexpr int SMEM_RING_F = MODE == 0 ? RING * TX2 : MODE == 1 ? RING * NDOG * TX2 : 0;
// per-pixel side data of the ring rows: the argmax (paper rule) or the mask
// of layers above the threshold (26-neighbour rule)
template <bool WIDE>
struct MaskT {
    using T = unsigned;
};
template <>
struct MaskT<true> {
    using T = unsigned long long;
};
using LMask = MaskT<(NDOG > 32)>::T;
constexpr int SMEM_RING_B = MODE == 0   ? ((RING * TX2 + 15) & ~15)
                            : MODE == 1 ? ((RING * TX2 * (int)sizeof(LMask) + 15) & ~15)
                                        : 0;
MK_HD constexpr int tc_kgp(int g) { return (RB + 2 * group_rmax(g) + 15) & ~15; }
// accumulator columns per level: RB rows, twice for the LoG (g and g'' rows)
constexpr int TC_P = LOG ? 2 : 1;
constexpr int TC_RC = RB * TC_P;
MK_HD constexpr int tc_ngp(int g) { return ((kGB(g + 1) - kGB(g)) * TC_RC + 15) & ~15; }
MK_HD constexpr int tc_colg(int g) {
    int o = 0;
    for (int j = 0; j < g; ++j) o += tc_ngp(j);
    return o;
}
// bytes of group g's B matrices (hi part then lo part) from the table start
MK_HD constexpr int tc_boff(int g) {
    int o = 0;
    for (int j = 0; j < g; ++j) o += 2 * 2 * tc_kgp(j) * tc_ngp(j);
    return o;
}
constexpr int TC_NCT = tc_colg(NGROUPS);  // TMEM columns per M tile
constexpr int TC_B_BYTES = TC ? tc_boff(NGROUPS) : 0;
MK_HD constexpr int tc_tcols() {
    int c = 32;
    while (c < TC_NMT * TC_NCT) c *= 2;
    return c;
}
constexpr int TC_TCOLS = tc_tcols();
constexpr int TC_CTRL = TC ? 128 : 0;  // mbarriers (one per group) and the TMEM address

// Two-pass kernel geometry: tiles of T2M computed rows (TY outputs and their
// two NMS neighbours) by TX2 computed columns.  Level l reads window rows
// [k0, k0 + KV) (K of its vertical product) and window columns [j0, j0 + NV)
// (its V columns, N of the vertical product, from an 8-aligned column: the
// horizontal product's column k is V column k + off); its horizontal product
// has K = KH window columns, of which the first TX2 + 2 R_l are used.
constexpr int T2M = 128;
MK_HD constexpr int t2_k0(int l) { return RMAX - kR(l); }
MK_HD constexpr int t2_j0(int l) { return (RMAX - kR(l)) & ~7; }
MK_HD constexpr int t2_off(int l) { return (RMAX - kR(l)) & 7; }
MK_HD constexpr int t2_need(int l) { return TX2 + 2 * kR(l); }
MK_HD constexpr int t2_kv(int l) { return (T2M + 2 * kR(l) + 15) & ~15; }
MK_HD constexpr int t2_nv(int l) { return (t2_off(l) + t2_need(l) + 15) & ~15; }
MK_HD constexpr int t2_kh(int l) { return (t2_need(l) + 15) & ~15; }
// blocks of 8 x 8 taps of level l's banded tap matrix (both products)
MK_HD constexpr int t2_s(int l) { return t2_kv(l) / 8 + 15; }
MK_HD constexpr int t2_maxf(int which) {
    int m = 0;
    for (int l = 0; l < NL; ++l) {
        const int v = which == 0   ? t2_nv(l)
                      : which == 1 ? t2_kh(l)
                      : which == 2 ? t2_s(l)
                      : which == 3 ? t2_k0(l) + t2_kv(l)
                                   : t2_j0(l) + t2_nv(l);
        m = v > m ? v : m;
    }
    return m;
}
constexpr int T2_NVMAX = t2_maxf(0);
constexpr int T2_KHMAX = t2_maxf(1);
constexpr int T2_SMAX = t2_maxf(2);
constexpr int T2_XIMG_R = T2M + 2 * RMAX;   // window rows holding image rows
constexpr int T2_XIMG_C = TX2 + 2 * RMAX;   // window columns holding image columns
constexpr int T2_XR = t2_maxf(3) > T2_XIMG_R ? t2_maxf(3) : T2_XIMG_R;  // + zero rows the K padding reads
constexpr int T2_XC = ((t2_maxf(4) > T2_XIMG_C ? t2_maxf(4) : T2_XIMG_C) + 7) & ~7;
// column group stride: 16 mod 128, so that eight lanes storing consecutive
// groups of one row hit distinct banks
constexpr int T2_XGSTR = ((16 * T2_XR + 127) / 128) * 128 + 16;
constexpr int T2_X_BYTES = TC2 ? (T2_XC / 8) * T2_XGSTR : 0;
constexpr int T2_TAB_PART = T2_SMAX * 128;  // one part (hi or lo) of a tap matrix
constexpr int T2_SBO_H = (T2_KHMAX / 8) * 128;
constexpr int T2_AH_PART = (T2M / 8) * T2_SBO_H;  // one part of the split V rows
constexpr int T2_OFF_TAB = (T2_X_BYTES + 127) & ~127;
constexpr int T2_NTAB = 4;                       // tap-matrix buffers (levels l - 1 .. l + 2)
constexpr int T2_OFF_AH = T2_OFF_TAB + (TC2 ? T2_NTAB * 2 * T2_TAB_PART : 0);
constexpr int T2_OFF_CTRL = T2_OFF_AH + (TC2 ? 2 * T2_AH_PART : 0);
// control block: mbarriers, tensor-memory address, fail flag, scan buffer,
// the window's column map
constexpr int T2_OFF_L26 = T2_OFF_CTRL + 512 + 4 * ((T2_XC + 3) & ~3);
// 26-neighbour rule: two exchange buffers of a layer's segment ends and
// lane-group boundary rows (parts x 2 x T2M floats; 8 x parts rows of a
// thread's columns + 4, so that the two boundary lanes' loads take distinct
// banks), then the per-pixel masks of kept layers (16 bits, [thread
// column][worker thread])
constexpr bool T2_L26 = TC2 && MODE == 1;
constexpr int T2_L26_CP = ((NT - 32) / 32) / 4;
constexpr int T2_L26_XB = 4 * (T2M * T2_L26_CP * 2 + 8 * (TX2 + 4 * T2_L26_CP));
constexpr int T2_SMEM = T2_OFF_L26 + (T2_L26 ? 2 * T2_L26_XB + 2 * TX2 * T2M : 0);
constexpr int T2_NW = NT - 32;                    // worker threads (the last warp issues)
constexpr int T2_DH = 2 * T2_NVMAX;               // tensor-memory column of the L buffers
constexpr int T2_LP = T2_DH + 2 * TX2;            // of the previous level's L (one copy)

constexpr int SMEM_BYTES =
    TC2 ? T2_SMEM
        : TC_WIN_BYTES + TC_B_BYTES + 4 * (SMEM_IN + SMEM_V + SMEM_RING_F) + SMEM_RING_B + 4 * 64 +
              TC_CTRL;
static_assert(!TC2 || ((MODE == 0 || MODE == 1) && !LOG), "two-pass kernel: detection with the DoG response");
static_assert(!T2_L26 || NL - 1 <= 16, "two-pass kernel, 26-neighbour rule: 16-bit layer masks");
static_assert(!TC2 || (TX2 % 16 == 0 && TX2 >= 16 && TX2 <= 128 && MHFD_TY2 == T2M &&
                       (NT == 288 || NT == 544) && TX2 % (4 * ((NT - 32) / 128)) == 0),
              "two-pass kernel geometry: 16-multiple strips up to 128, tiles of 128 rows, 8 or 16 worker warps");
static_assert(!TC2 || T2_LP + TX2 <= 512, "two-pass kernel: tensor memory columns");
static_assert(!TC2 || T2_NVMAX <= 256, "two-pass kernel: N of the vertical product");
// the tile-end maxima test's exchange arrays (segment edges, boundary rows,
// counts and their prefix), then its stashed responses and argmaxes, in the
// split rows' space
constexpr int T2_NMS_VALS = 8192;
static_assert(!TC2 || (4 * (T2M * 2 * 2 + 8 * TX2 + 2 * T2M * 2) <= T2_NMS_VALS &&
                       T2_NMS_VALS + 5 * TX2 * T2M <= 2 * T2_AH_PART),
              "two-pass kernel: tile-end maxima space");

static_assert(TX2 % 4 == 0, "tile width must be a multiple of 4");
static_assert(TY >= 1, "tile height");
static_assert(BROWS >= WIN, "the input window must hold one step");
static_assert(NT % 32 == 0 && NT <= 1024, "threads per block");
static_assert((MODE == 3 || LOG ? NL >= 1 : NL >= 2) && NL <= 64, "levels");
static_assert(!LOG || MODE <= 1, "the LoG response is a detection mode");
static_assert(kGB(0) == 0 && kGB(NGROUPS) == NL, "level groups");
static_assert(!TC || ((MODE == 0 || (MODE == 1 && !LOG)) && (RB == 4 || RB == 8) && NT >= 128),
              "tensor-core vertical pass");
static_assert(!TC || TC_NMT * TC_NCT <= 512, "tensor memory columns");
static_assert(!TC || BROWS >= WIN + 2 * RB + 16, "window rows of the tensor-core pass");
static_assert(!TC || NGROUPS <= 12, "one mbarrier per group in the control block");
static_assert(HR == 1 || (HR == 2 && RB % 2 == 0 && MODE <= 1), "two-row horizontal items");
static_assert(HW == 4 || (HW == 2 && HR == 1), "two-output horizontal items have one row");

struct KParams {
    MhfdKHeader h;
};

constexpr int NSOFT = MODE == 2 ? NDOG : 1;

// state of one row of a horizontal item (four outputs) across the levels
struct HRowState {
    float lp[4];  // L of the previous level
    float m[4];   // running max over scales
    int a[4];     // its first argmax
    // 26-neighbour rule: layers whose response is above the threshold and
    // not below either scale neighbour at the same pixel (the only layers
    // whose 3x3x3 test can pass), and the previous layer's response
    LMask mk[4];
    float dp[4];
};
struct HState {
    HRowState rw[HR];
    // soft-score forward: running sums over the march of sigmoid((D_i -
    // tau) / T) at this item's interior output pixels, per layer
    float soft[NSOFT];
};

// Image index of a position outside [0, n): reflect ("d c b a | a b c d |
// d c b a", the default) or periodic (MHFD_BOUNDARY 1, the circular
// convolution of the paper's Fourier formulation).
__device__ __forceinline__ int reflect_idx_(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    if constexpr (MHFD_BOUNDARY == 1) {
        const int m = i % n;
        return m < 0 ? m + n : m;
    } else {
        const int p = 2 * n;
        int m = i % p;
        if (m < 0) m += p;
        return m < n ? m : p - 1 - m;
    }
}
__device__ __forceinline__ int reflect_idx(int i, int n) {
    const int k = reflect_idx_(i, n);
    return mk_ok((unsigned)k < (unsigned)n) ? k : 0;
}

// ---------------------------------------------------------------- 1. load

// raw pixel bits (the stretch is applied when the value is stored, so that
// a prefetched load is not waited for until then)
template <int DT>
__device__ __forceinline__ unsigned raw_px(const char *row, int gx) {
    if (DT == 0) return __ldg(reinterpret_cast<const unsigned char *>(row) + gx);
    if (DT == 1) return __ldg(reinterpret_cast<const unsigned short *>(row) + gx);
    return __float_as_uint(__ldg(reinterpret_cast<const float *>(row) + gx));
}

template <int DT>
__device__ __forceinline__ float stretch_px(unsigned raw, const MhfdStretch &st) {
    if constexpr (MODE == 3) return __uint_as_float(raw);  // a plane, taken as it is
    if (DT == 2) {
        float u = (__uint_as_float(raw) - st.lo) * st.inv;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        return u + st.off;
    }
    const int v = min(max((int)raw, st.lo_i), st.hi_i);
    return fmaf((float)(v - st.lo_i), st.inv, st.off);
}

// Strip geometry of one march: input row i of the window is image row
// reflect(yin + i); input column c is image column reflect(xin + c).
struct Strip {
    const char *img;
    long long pitch;
    int H, W, dtype;
    int xin, yin;
};

// Load input rows [r0, r1) into window rows [r0 - base, r1 - base), LB row
// loads in flight per thread.
template <int DT>
__device__ __forceinline__ void load_rows_t(const Strip &sp, const MhfdStretch &st, float *s_in,
                                            int r0, int r1, int base) {
    constexpr int LB = 16;
    for (int c = threadIdx.x; c < WEXT; c += NT) {
        const int gx = reflect_idx(sp.xin + c, sp.W);
        float *dst = s_in + c;
#pragma unroll 1
        for (int r = r0; r < r1; r += LB) {
            unsigned v[LB];
#pragma unroll
            for (int e = 0; e < LB; ++e)
                if (r + e < r1)
                    v[e] = raw_px<DT>(sp.img + (long long)reflect_idx(sp.yin + r + e, sp.H) * sp.pitch,
                                      gx);
#pragma unroll
            for (int e = 0; e < LB; ++e)
                if (r + e < r1 && mk_ok((unsigned)(r + e - base) < (unsigned)BROWS))
                    dst[(r + e - base) * WEXTP] = stretch_px<DT>(v[e], st);
        }
    }
}

__device__ __forceinline__ void load_rows(const Strip &sp, const MhfdStretch &st, float *s_in,
                                          int r0, int r1, int base) {
    if (sp.dtype == 0)
        load_rows_t<0>(sp, st, s_in, r0, r1, base);
    else if (sp.dtype == 1)
        load_rows_t<1>(sp, st, s_in, r0, r1, base);
    else
        load_rows_t<2>(sp, st, s_in, r0, r1, base);
}

// The RB input rows of the next step, held in registers across a step.
struct Prefetch {
    unsigned v[NT_COLS][RB];

    template <int DT>
    __device__ __forceinline__ void issue_t(const Strip &sp, int r0) {
#pragma unroll
        for (int k = 0; k < NT_COLS; ++k) {
            const int c = threadIdx.x + k * NT;
            if (c < WEXT) {
                const int gx = reflect_idx(sp.xin + c, sp.W);
#pragma unroll
                for (int e = 0; e < RB; ++e)
                    v[k][e] = raw_px<DT>(
                        sp.img + (long long)reflect_idx(sp.yin + r0 + e, sp.H) * sp.pitch, gx);
            }
        }
    }
    __device__ __forceinline__ void issue(const Strip &sp, int r0) {
        if (sp.dtype == 0)
            issue_t<0>(sp, r0);
        else if (sp.dtype == 1)
            issue_t<1>(sp, r0);
        else
            issue_t<2>(sp, r0);
    }
    template <int DT>
    __device__ __forceinline__ void store_t(const MhfdStretch &st, float *s_in, int prow) const {
#pragma unroll
        for (int k = 0; k < NT_COLS; ++k) {
            const int c = threadIdx.x + k * NT;
            if (c < WEXT) {
#pragma unroll
                for (int e = 0; e < RB; ++e)
                    if (mk_ok((unsigned)(prow + e) < (unsigned)BROWS))
                        s_in[(prow + e) * WEXTP + c] = stretch_px<DT>(v[k][e], st);
            }
        }
    }
    __device__ __forceinline__ void store(int dtype, const MhfdStretch &st, float *s_in,
                                          int prow) const {
        if (dtype == 0)
            store_t<0>(st, s_in, prow);
        else if (dtype == 1)
            store_t<1>(st, s_in, prow);
        else
            store_t<2>(st, s_in, prow);
    }
};

// Move window rows [from, from + n) to [0, n) (each thread its own columns;
// the destination lies below the source, batches are read before written).
__device__ __forceinline__ void shift_window(float *s_in, int from, int n) {
    constexpr int SB = 8;
    if (!mk_ok(from >= 0 && n >= 0 && from + n <= BROWS)) return;
    for (int c = threadIdx.x; c < WEXT; c += NT) {
        float *col = s_in + c;
#pragma unroll 1
        for (int r = 0; r < n; r += SB) {
            float v[SB];
#pragma unroll
            for (int e = 0; e < SB; ++e)
                if (r + e < n) v[e] = col[(from + r + e) * WEXTP];
#pragma unroll
            for (int e = 0; e < SB; ++e)
                if (r + e < n) col[(r + e) * WEXTP] = v[e];
        }
    }
}


// ----------------------------------------- tensor-core vertical pass (TC)
//
// V_l(y0 + j, c) = sum_k g_l[k - j - RG] x(y0 + RMAX - RG + k, c) for the
// levels l of group G is the product of the window (M = columns, K = rows,
// MN-major) with a banded tap matrix B_G (K x N, N = (level, row j)), built
// once per block: taps scaled by TC_S and split into fp16 hi and lo parts,
// so that the two products add up to the f32 tap to about 2^-22 while the
// window values are exact.  One elected thread issues the MMAs
// (tcgen05.mma, kind::f16, f32 accumulators in tensor memory) for the next
// step of a group as soon as this step's results of the group have been
// read out, so they run under the horizontal passes; the block reads each
// group's accumulators back with tcgen05.ld (lane = column) and writes them
// unscaled as the V rows the horizontal pass reads: the stretch affine
// (acc / TC_S) inv + (c0 - lo) inv + off is a scale, applied to the response,
// plus an offset that the DoG difference and the zero-sum second-difference
// taps remove.  All waits are bounded: a wait that gives up
// sets h.flag and the block carries on (the results are then reported as
// unreliable by the host).

__device__ const float mk_taps_rt[NTAPS] = {MHFD_TAPS};
__device__ const float mk_taps2_rt[] = {MHFD_TAPS2};
struct TcTab {
    int r[NL];
    int off[NL];
    int off2[NL];
};
MK_HD constexpr TcTab tc_tab() {
    TcTab t{};
    for (int l = 0; l < NL; ++l) {
        t.r[l] = kR(l);
        t.off[l] = tapoff(l);
        t.off2[l] = tapoff2(l);
    }
    return t;
}
__device__ const TcTab mk_tctab = tc_tab();

__device__ __forceinline__ unsigned short f2h_rn(float f) {
    unsigned short h;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return h;
}
__device__ __forceinline__ float h2f(unsigned short h) {
    float f;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
    return f;
}
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// stretch of one image for the tensor-core pass
struct TcStretch {
    int lo, hi, c0;
    float a;  // stretched units per unit of the MMA sums
};
__device__ __forceinline__ TcStretch tc_stretch(const MhfdStretch &st) {
    TcStretch t;
    t.lo = st.lo_i;
    t.hi = st.hi_i;
    t.c0 = (st.lo_i + st.hi_i) >> 1;
    t.a = st.inv * (1.0f / TC_S);
    return t;
}
// uint8, or uint16 whose stretch range keeps |x| <= 2048
__device__ __forceinline__ bool tc_narrow(int dtype, const MhfdStretch &st) {
    return dtype == 0 || (dtype == 1 && st.hi_i - st.lo_i <= 4095);
}
__device__ __forceinline__ unsigned short tc_px(unsigned raw, const TcStretch &ts) {
    const int v = min(max((int)raw, ts.lo), ts.hi) - ts.c0;
    return f2h_rn((float)v);
}
__device__ __forceinline__ void tc_put(unsigned char *win, int row, int c, unsigned short v) {
    if (!mk_ok((unsigned)row < (unsigned)BROWS && (unsigned)c < (unsigned)TC_WT)) return;
    *reinterpret_cast<unsigned short *>(win + (c >> 3) * TC_GSTR + row * 16 + (c & 7) * 2) = v;
}

// Input rows [r0, r1) into window rows [r0, r1) (the start of a march).
template <int DT>
__device__ __forceinline__ void tc_load_rows_t(const Strip &sp, const TcStretch &ts,
                                               unsigned char *win, int r0, int r1) {
    constexpr int LB = 16;
    for (int c = threadIdx.x; c < WEXT; c += NT) {
        const int gx = reflect_idx(sp.xin + c, sp.W);
#pragma unroll 1
        for (int r = r0; r < r1; r += LB) {
            unsigned v[LB];
#pragma unroll
            for (int e = 0; e < LB; ++e)
                if (r + e < r1)
                    v[e] = raw_px<DT>(sp.img + (long long)reflect_idx(sp.yin + r + e, sp.H) * sp.pitch,
                                      gx);
#pragma unroll
            for (int e = 0; e < LB; ++e)
                if (r + e < r1) tc_put(win, r + e, c, tc_px(v[e], ts));
        }
    }
}
__device__ __forceinline__ void tc_load_rows(const Strip &sp, const TcStretch &ts,
                                             unsigned char *win, int r0, int r1) {
    if (sp.dtype == 0)
        tc_load_rows_t<0>(sp, ts, win, r0, r1);
    else
        tc_load_rows_t<1>(sp, ts, win, r0, r1);
}

// Move window rows [from, from + n) to [0, n): one thread per column group
// walks its rows upwards, eight at a time (read before written).
__device__ __forceinline__ void tc_shift(unsigned char *win, int from, int n) {
    if (!mk_ok(from >= 0 && n >= 0 && from + n <= BROWS)) return;
    for (int cg = threadIdx.x; cg < TC_CGL; cg += NT) {
        uint4 *col = reinterpret_cast<uint4 *>(win + cg * TC_GSTR);
#pragma unroll 1
        for (int r = 0; r < n; r += 8) {
            uint4 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (r + e < n) v[e] = col[from + r + e];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (r + e < n) col[r + e] = v[e];
        }
    }
}

// Zero the window (rows and columns the MMAs read but no image row fills
// must hold finite values) and build the B matrices: K-major, core matrices
// of 8 N-rows x 8 K-values (128 bytes), K-adjacent core matrices 128 bytes
// apart, N-adjacent ones (kgp / 8) * 128 bytes apart.
__device__ __forceinline__ void tc_setup_smem(unsigned char *win, unsigned char *btab) {
    for (int i = threadIdx.x; i < TC_WIN_BYTES / 16; i += NT)
        reinterpret_cast<uint4 *>(win)[i] = make_uint4(0u, 0u, 0u, 0u);
    unsigned short *hb = reinterpret_cast<unsigned short *>(btab);
    for (int g = 0; g < NGROUPS; ++g) {
        const int kgp = tc_kgp(g), ngp = tc_ngp(g), rg = group_rmax(g);
        const int lb = kGB(g), ng = kGB(g + 1) - lb;
        const int part = kgp * ngp;
        unsigned short *p0 = hb + tc_boff(g) / 2;
        for (int q = threadIdx.x; q < part; q += NT) {
            const int blk = q >> 6, e = q & 63;
            const int n = (blk / (kgp / 8)) * 8 + (e >> 3);
            const int k = (blk % (kgp / 8)) * 8 + (e & 7);
            // column n = level li x TC_RC + part x RB + row j (part 1: the
            // LoG's second-difference taps, radius R + 1)
            const int li = n / TC_RC, rem = n - li * TC_RC;
            const int part2 = rem / RB, j = rem - part2 * RB;
            float v = 0.0f;
            if (li < ng) {
                const int l = lb + li;
                int d = k - j - rg;
                d = d < 0 ? -d : d;
                if (!part2 && d <= mk_tctab.r[l]) v = mk_taps_rt[mk_tctab.off[l] + d] * TC_S;
                if (part2 && d <= mk_tctab.r[l] + 1) v = mk_taps2_rt[mk_tctab.off2[l] + d] * TC_S;
            }
            const unsigned short hi = f2h_rn(v);
            p0[q] = hi;
            p0[part + q] = f2h_rn(v - h2f(hi));
        }
    }
}

// shared-memory matrix descriptor: no swizzle, start / leading (K) / stride
// (M or N) byte offsets in 16-byte units, descriptor version 1
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) |
           ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: f32 accumulator, f16 A and B, A
// MN-major, B K-major, N >> 3 and M >> 4
MK_HD constexpr unsigned tc_idesc(int n) {
    return (1u << 4) | (1u << 15) | ((unsigned)(n >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}

// The thread that issues the MMAs: lane 0 of the first warp without a
// horizontal item when there is one (its issue then runs beside the
// horizontal passes of the other warps), else thread 0.
constexpr int TC_ISSUER = NTW < NT                               ? NTW
                          : ((HITEMS + 31) / 32) * 32 < NT ? ((HITEMS + 31) / 32) * 32
                                                           : 0;

struct TcState {
    unsigned tmem;   // tensor-memory base (lane 0, first column)
    unsigned win;    // shared addresses of the window, the B table, the mbarriers
    unsigned btab;
    unsigned bar;
    unsigned ph;     // expected phase parity per group (bit G)
    bool issuer;
};

// The MMAs of group G for the step whose first input row is window row row0.
template <int G>
__device__ __forceinline__ void tc_issue(const TcState &tc, int row0) {
    constexpr int NK = tc_kgp(G) / 16;
    constexpr unsigned IDESC = tc_idesc(tc_ngp(G));
    constexpr unsigned PART = 2u * tc_kgp(G) * tc_ngp(G);
    // (a failed check issues no MMA but still commits, so the waits end)
    const bool rows_ok = mk_ok(row0 + RMAX - group_rmax(G) >= 0 &&
                               row0 + RMAX - group_rmax(G) + tc_kgp(G) <= BROWS);
    const unsigned long long a0 =
        tc_desc(tc.win + (unsigned)(row0 + RMAX - group_rmax(G)) * 16u, 128u, (unsigned)TC_GSTR);
    const unsigned long long b0 =
        tc_desc(tc.btab + (unsigned)tc_boff(G), 128u, (unsigned)(tc_kgp(G) / 8) * 128u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
    for (int t = 0; t < (rows_ok ? TC_NMT : 0); ++t) {
        const unsigned d = tc.tmem + (unsigned)(t * TC_NCT + tc_colg(G));
        const unsigned long long at = a0 + (unsigned long long)((t * 16 * TC_GSTR) >> 4);
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const unsigned long long a = at + (unsigned long long)(kk * 16);
                const unsigned long long b = b0 + (unsigned long long)((p * PART + kk * 256) >> 4);
                const unsigned acc = (kk | p) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(d),
                    "l"(a), "l"(b), "r"(IDESC), "r"(acc)
                    : "memory");
            }
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc.bar + 8u * G)
                 : "memory");
}

__device__ __forceinline__ bool tc_try(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
        "selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the MMAs of group G to complete, at most 2 s of global time (as
// the prune's settle loop; far beyond any MMA batch, and long enough that a
// block preempted by time slicing does not give up early).
__device__ __forceinline__ void tc_wait(const MhfdKHeader &h, const TcState &tc, int g) {
    const unsigned bar = tc.bar + 8u * g, par = (tc.ph >> g) & 1u;
    if (tc_try(bar, par)) return;
    const unsigned long long t0 = gtimer();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 256; ++i)
            if (tc_try(bar, par)) return;
        if (gtimer() - t0 > 2000000000ull) break;
    }
    if (h.flag) atomicOr(h.flag, 1);
}

// four / eight accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tc_ld4(unsigned addr, unsigned *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr)
                 : "memory");
}
__device__ __forceinline__ void tc_ld8(unsigned addr, unsigned *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(addr)
        : "memory");
}
// the TC_RC accumulator columns of one level (rows j = 0 .. RB-1, then for
// the LoG the second-difference rows)
__device__ __forceinline__ void tc_ld_rows(unsigned addr, unsigned (&r)[TC_RC]) {
#pragma unroll
    for (int c = 0; c + 8 <= TC_RC; c += 8) tc_ld8(addr + (unsigned)c, r + c);
    if constexpr (TC_RC % 8 == 4) tc_ld4(addr + (unsigned)(TC_RC - 4), r + TC_RC - 4);
}

// the RB prefetched rows into window rows [prow, prow + RB)
__device__ __forceinline__ void tc_store_prefetch(const Prefetch &pf, const TcStretch &ts,
                                                  unsigned char *win, int prow) {
#pragma unroll
    for (int k = 0; k < NT_COLS; ++k) {
        const int c = threadIdx.x + k * NT;
        if (c < WEXT) {
#pragma unroll
            for (int e = 0; e < RB; ++e) tc_put(win, prow + e, c, tc_px(pf.v[k][e], ts));
        }
    }
}

// the loaded registers are only read after tcgen05.wait::ld: this empty
// statement (ordered after the wait like every volatile asm) redefines them
__device__ __forceinline__ void tc_regs_ready(unsigned (&r)[TC_RC]) {
#pragma unroll
    for (int j = 0; j < TC_RC; j += 4)
        asm volatile("" : "+r"(r[j]), "+r"(r[j + 1]), "+r"(r[j + 2]), "+r"(r[j + 3]));
}

template <int G, int LI>
__device__ __forceinline__ void tc_ld_levels(unsigned taddr, unsigned (*r)[TC_RC]) {
    if constexpr (LI < kGB(G + 1) - kGB(G)) {
        tc_ld_rows(taddr + (unsigned)(LI * TC_RC), r[LI]);
        tc_ld_levels<G, LI + 1>(taddr, r);
    }
}
template <int G, int LI>
__device__ __forceinline__ void tc_st_levels(float *__restrict__ s_v, unsigned (*r)[TC_RC], int c,
                                             const TcStretch &ts) {
    if constexpr (LI < kGB(G + 1) - kGB(G)) {
        constexpr int L = kGB(G) + LI;
        tc_regs_ready(r[LI]);
        const int cc = c - (RMAX - kRH(L));
        if (cc >= 0 && cc < TX2 + 2 * kRH(L)) {
            // the raw MMA sums (the horizontal pass applies the scale), and
            // the LoG's g'' (*)_y I row beside them
#pragma unroll
            for (int pt = 0; pt < TC_P; ++pt) {
                if constexpr (HR == 2) {
#pragma unroll
                    for (int j = 0; j < RB; j += 2)
                        if (mk_ok((unsigned)(vidx(L, pt, j, cc) + 1) < (unsigned)SMEM_V))
                            *reinterpret_cast<float2 *>(s_v + vidx(L, pt, j, cc)) = make_float2(
                                __uint_as_float(r[LI][pt * RB + j]),
                                __uint_as_float(r[LI][pt * RB + j + 1]));
                } else {
#pragma unroll
                    for (int j = 0; j < RB; ++j)
                        if (mk_ok((unsigned)vidx(L, pt, j, cc) < (unsigned)SMEM_V))
                            s_v[vidx(L, pt, j, cc)] = __uint_as_float(r[LI][pt * RB + j]);
                }
            }
        }
        tc_st_levels<G, LI + 1>(s_v, r, c, ts);
    }
}

// Read group G's accumulators and write the V rows of its levels: warp w
// reads tensor-memory lanes 32 (w % 4) .. + 31 (window columns 128 t + lane)
// of the M tiles t = w / 4, w / 4 + NT / 128, ...
template <int G>
__device__ __forceinline__ void tc_read(const TcState &tc, float *s_v, const TcStretch &ts) {
    constexpr int NG = kGB(G + 1) - kGB(G);
    constexpr int NWG = NT / 128;  // a last partial warpgroup does not read
    const int warp = threadIdx.x >> 5, q = warp & 3;
    if ((warp >> 2) >= NWG) return;
    const int c0 = 32 * q + (threadIdx.x & 31);
#pragma unroll 1
    for (int t = warp >> 2; t < TC_NMT; t += NWG) {
        const unsigned taddr =
            tc.tmem + ((unsigned)(32 * q) << 16) + (unsigned)(t * TC_NCT + tc_colg(G));
        unsigned r[NG][TC_RC];
        tc_ld_levels<G, 0>(taddr, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tc_st_levels<G, 0>(s_v, r, 128 * t + c0, ts);
    }
}

// Fold step K of the vertical pass for the levels L.. of group G: every
// level whose radius reaches K takes tap K times the folded sum (and, for
// the LoG, every level whose radius + 1 reaches K its second-difference
// tap K into a2).
template <int G, int K, int L>
__device__ __forceinline__ void vlev(float sum, float *a, float *a2) {
    constexpr int LB = kGB(G);
    constexpr int NG = kGB(G + 1) - LB;
    if constexpr (L < NG) {
        if constexpr (K <= kR(LB + L)) a[L] = fmaf(tap<tapoff(LB + L) + K>(), sum, a[L]);
        if constexpr (LOG && K <= kR(LB + L) + 1)
            a2[L] = fmaf(tap2<tapoff2(LB + L) + K>(), sum, a2[L]);
        vlev<G, K, L + 1>(sum, a, a2);
    }
}

template <int G, int L>
__device__ __forceinline__ void vinit(float x, float *a, float *a2) {
    constexpr int LB = kGB(G);
    constexpr int NG = kGB(G + 1) - LB;
    if constexpr (L < NG) {
        a[L] = tap<tapoff(LB + L)>() * x;
        if constexpr (LOG) a2[L] = tap2<tapoff2(LB + L)>() * x;
        vinit<G, L + 1>(x, a, a2);
    }
}

template <int G>
MK_HD constexpr int ng2() { return LOG ? kGB(G + 1) - kGB(G) : 1; }

template <int G, int ROWS, int K>
__device__ __forceinline__ void vstep(const float *colp, float (*acc)[kGB(G + 1) - kGB(G)],
                                      float (*acc2)[ng2<G>()]) {
    if constexpr (K <= group_rmax(G)) {
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const float sum = colp[(j + K) * WEXTP] + colp[(j - K) * WEXTP];
            vlev<G, K, 0>(sum, acc[j], acc2[j]);
        }
        vstep<G, ROWS, K + 1>(colp, acc, acc2);
    }
}

// V_l(o0 + j, c) for the ROWS rows starting at step row o0 and every level l
// of group G (for the LoG also g''_l (*)_y I, stored after V_l).  `win` is
// the window row of the step's first input row: step row o sits at window
// row o + RMAX.
template <int G, int ROWS>
__device__ __forceinline__ void vcol(const float *__restrict__ win, float *__restrict__ s_v, int c,
                                     int o0) {
    constexpr int LB = kGB(G);
    constexpr int LE = kGB(G + 1);
    constexpr int NG = LE - LB;
    float acc[ROWS][NG];
    float acc2[ROWS][ng2<G>()];
    const float *colp = win + (o0 + RMAX) * WEXTP + c;
#pragma unroll
    for (int j = 0; j < ROWS; ++j) vinit<G, 0>(colp[j * WEXTP], acc[j], acc2[j]);
    vstep<G, ROWS, 1>(colp, acc, acc2);
#pragma unroll
    for (int l = 0; l < NG; ++l) {
        const int cc = c - (RMAX - kRH(LB + l));
        if (cc >= 0 && cc < TX2 + 2 * kRH(LB + l)) {
            if constexpr (HR == 2 && ROWS % 2 == 0) {
#pragma unroll
                for (int j = 0; j < ROWS; j += 2) {
                    if (mk_ok((unsigned)(vidx(LB + l, LOG ? 1 : 0, o0 + j, cc) + 1) <
                              (unsigned)SMEM_V)) {
                        *reinterpret_cast<float2 *>(s_v + vidx(LB + l, 0, o0 + j, cc)) =
                            make_float2(acc[j][l], acc[j + 1][l]);
                        if constexpr (LOG)
                            *reinterpret_cast<float2 *>(s_v + vidx(LB + l, 1, o0 + j, cc)) =
                                make_float2(acc2[j][l], acc2[j + 1][l]);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    if (!mk_ok((unsigned)vidx(LB + l, LOG ? 1 : 0, o0 + j, cc) < (unsigned)SMEM_V))
                        continue;
                    s_v[vidx(LB + l, 0, o0 + j, cc)] = acc[j][l];
                    if constexpr (LOG) s_v[vidx(LB + l, 1, o0 + j, cc)] = acc2[j][l];
                }
            }
        }
    }
}

template <int G, int PART>
struct VParts {
    static __device__ __forceinline__ void run(const float *win, float *s_v, int c) {
        constexpr int ROWS = (RB - 4 * PART) < 4 ? (RB - 4 * PART) : 4;
        vcol<G, ROWS>(win, s_v, c, 4 * PART);
        VParts<G, PART + 1>::run(win, s_v, c);
    }
};
template <int G>
struct VParts<G, NPARTS> {
    static __device__ __forceinline__ void run(const float *, float *, int) {}
};

template <int G>
__device__ __forceinline__ void vpass(const float *win, float *s_v) {
    constexpr int RG = group_rmax(G);
    constexpr int CB = RMAX - RG;
    constexpr int CE = RMAX + TX2 + RG;
#pragma unroll 1
    for (int c = CB + threadIdx.x; c < CE; c += NT) VParts<G, 0>::run(win, s_v, c);
}

// ----------------------------------------------------- 3. horizontal pass

// value number M of the window (which starts OFF values before the first
// output's) feeds output U with tap |M - U - R - OFF| of the Gaussian taps,
// or of the second-difference taps when T2
template <int R, int TO, int M, int U, int OFF, bool T2>
__device__ __forceinline__ void hacc1(float v, float (&a)[4]) {
    constexpr int k = M - U - R - OFF;
    if constexpr (k >= -R && k <= R) {
        if constexpr (T2)
            a[U] = fmaf(tap2<TO + (k < 0 ? -k : k)>(), v, a[U]);
        else
            a[U] = fmaf(tap<TO + (k < 0 ? -k : k)>(), v, a[U]);
    }
}

template <int R, int TO, int M, int OFF, bool T2>
__device__ __forceinline__ void hacc(float v, float (&a)[4]) {
    hacc1<R, TO, M, 0, OFF, T2>(v, a);
    hacc1<R, TO, M, 1, OFF, T2>(v, a);
    hacc1<R, TO, M, 2, OFF, T2>(v, a);
    hacc1<R, TO, M, 3, OFF, T2>(v, a);
}

template <int R, int TO, int M4, int OFF, bool T2>
struct HQuads {
    static __device__ __forceinline__ void run(const float4 *w, float (&a)[4]) {
        const float4 v = w[M4];
        hacc<R, TO, 4 * M4 + 0, OFF, T2>(v.x, a);
        hacc<R, TO, 4 * M4 + 1, OFF, T2>(v.y, a);
        hacc<R, TO, 4 * M4 + 2, OFF, T2>(v.z, a);
        hacc<R, TO, 4 * M4 + 3, OFF, T2>(v.w, a);
        HQuads<R, TO, M4 - 1, OFF, T2>::run(w, a);
    }
};
template <int R, int TO, int OFF, bool T2>
struct HQuads<R, TO, -1, OFF, T2> {
    static __device__ __forceinline__ void run(const float4 *, float (&)[4]) {}
};

// The same sums with packed two-lane FMAs (sm_100 and later): outputs
// (0, 1) and (2, 3) of the item form two lane pairs, and the window values
// M, M + 1 feed both lanes of a pair with one tap, |M - R - OFF| for the
// first and |M - 2 - R - OFF| for the second.  Pairs at even M are halves of
// the loaded float4s; pairs at odd M straddle them.
template <int R, int TO, int M, int OFF, bool T2>
__device__ __forceinline__ void hpk(float2 v, float2 (&a)[2]) {
    constexpr int k0 = M - R - OFF, k1 = M - 2 - R - OFF;
    constexpr int a0 = k0 < 0 ? -k0 : k0, a1 = k1 < 0 ? -k1 : k1;
    if constexpr (a0 <= R) {
        constexpr float t = T2 ? kTap2(TO + a0) : kTap(TO + a0);
        a[0] = __ffma2_rn(make_float2(t, t), v, a[0]);
    }
    if constexpr (a1 <= R) {
        constexpr float t = T2 ? kTap2(TO + a1) : kTap(TO + a1);
        a[1] = __ffma2_rn(make_float2(t, t), v, a[1]);
    }
}

template <int R, int TO, int NQ, int OFF, bool T2, int I>
struct HQuadsP {
    static __device__ __forceinline__ void run(const float4 *w, float2 (&a)[2], float prevw) {
        const float4 v = w[I];
        if constexpr (I > 0) hpk<R, TO, 4 * I - 1, OFF, T2>(make_float2(prevw, v.x), a);
        hpk<R, TO, 4 * I, OFF, T2>(make_float2(v.x, v.y), a);
        hpk<R, TO, 4 * I + 1, OFF, T2>(make_float2(v.y, v.z), a);
        hpk<R, TO, 4 * I + 2, OFF, T2>(make_float2(v.z, v.w), a);
        HQuadsP<R, TO, NQ, OFF, T2, I + 1>::run(w, a, v.w);
    }
};
template <int R, int TO, int NQ, int OFF, bool T2>
struct HQuadsP<R, TO, NQ, OFF, T2, NQ> {
    // the pair at 4 NQ - 1 would need the next float4: it feeds no output
    static_assert(4 * NQ - 1 > 2 * R + 2 + OFF, "window of the packed horizontal pass");
    static __device__ __forceinline__ void run(const float4 *, float2 (&)[2], float) {}
};

template <int R, int TO, int NQ, int OFF, bool T2>
__device__ __forceinline__ void hquads(const float4 *w, float (&a)[4]) {
    if constexpr (HPACK) {
        float2 p[2] = {make_float2(a[0], a[1]), make_float2(a[2], a[3])};
        HQuadsP<R, TO, NQ, OFF, T2, 0>::run(w, p, 0.0f);
        a[0] = p[0].x;
        a[1] = p[0].y;
        a[2] = p[1].x;
        a[3] = p[1].y;
    } else {
        HQuads<R, TO, NQ - 1, OFF, T2>::run(w, a);
    }
}

// one row of a horizontal item
struct HRowCtx {
    int r;          // chunk row
    int slot;       // ring slot of row r
    int gy;         // image row
    bool inb[4];    // output inside the image
    bool inter[4];  // output inside the tile interior and the image (stored)
};
struct HCtx {
    int q;          // float4 chunk (outputs 4q .. 4q+3)
    int j0;         // first step row of the item
    int gx0;        // image column of output 4q
    HRowCtx rw[HR];
};

// Two-row items: window column M (a float2 of both rows' values) feeds
// output U of both rows with tap |M - U - R - OFF| (of the second-difference
// taps when T2): one packed two-lane FMA.
template <int R, int TO, int M, int U, int OFF, bool T2>
__device__ __forceinline__ void hacc2u(float2 v, float2 (&a)[4]) {
    constexpr int k = M - U - R - OFF;
    if constexpr (k >= -R && k <= R) {
        constexpr float t = T2 ? kTap2(TO + (k < 0 ? -k : k)) : kTap(TO + (k < 0 ? -k : k));
        a[U] = __ffma2_rn(make_float2(t, t), v, a[U]);
    }
}
template <int R, int TO, int M, int OFF, bool T2>
__device__ __forceinline__ void hacc2(float2 v, float2 (&a)[4]) {
    hacc2u<R, TO, M, 0, OFF, T2>(v, a);
    hacc2u<R, TO, M, 1, OFF, T2>(v, a);
    hacc2u<R, TO, M, 2, OFF, T2>(v, a);
    hacc2u<R, TO, M, 3, OFF, T2>(v, a);
}
// Columns in the order of the one-row pass (quads of four columns
// descending, columns ascending within a quad), so that each lane sums
// exactly as the one-row pass does.  `w` points at the item's column 4q of
// the level row in the residue-ordered pair layout (S = extp / 4 entries
// per residue class): window column M of the item is w[(M % 4) S + M / 4].
template <int R, int TO, int Q, int OFF, bool T2, int S>
struct HQuads2 {
    static __device__ __forceinline__ void run(const float2 *w, float2 (&a)[4]) {
        hacc2<R, TO, 4 * Q + 0, OFF, T2>(w[0 * S + Q], a);
        hacc2<R, TO, 4 * Q + 1, OFF, T2>(w[1 * S + Q], a);
        hacc2<R, TO, 4 * Q + 2, OFF, T2>(w[2 * S + Q], a);
        hacc2<R, TO, 4 * Q + 3, OFF, T2>(w[3 * S + Q], a);
        HQuads2<R, TO, Q - 1, OFF, T2, S>::run(w, a);
    }
};
template <int R, int TO, int OFF, bool T2, int S>
struct HQuads2<R, TO, -1, OFF, T2, S> {
    static __device__ __forceinline__ void run(const float2 *, float2 (&)[4]) {}
};

// Two-output items: window column M feeds outputs 0 and 1; float2 loads (two
// columns), descending like the four-output pass.
template <int R, int TO, int P, int OFF, bool T2>
struct HPairs {
    static __device__ __forceinline__ void run(const float2 *w, float (&a)[4]) {
        const float2 v = w[P];
        hacc1<R, TO, 2 * P, 0, OFF, T2>(v.x, a);
        hacc1<R, TO, 2 * P, 1, OFF, T2>(v.x, a);
        hacc1<R, TO, 2 * P + 1, 0, OFF, T2>(v.y, a);
        hacc1<R, TO, 2 * P + 1, 1, OFF, T2>(v.y, a);
        HPairs<R, TO, P - 1, OFF, T2>::run(w, a);
    }
};
template <int R, int TO, int OFF, bool T2>
struct HPairs<R, TO, -1, OFF, T2> {
    static __device__ __forceinline__ void run(const float2 *, float (&)[4]) {}
};

// The horizontal sums of level L for the item's outputs: a[rr][u] for row rr.
// `vbase` is the item's first row in the V rows (row pair for two-row items).
template <int L>
__device__ __forceinline__ void hsums(const float *vbase, int q, float (&a)[HR][4]) {
    constexpr int R = kR(L);
    if constexpr (HR == 2) {
        float2 p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = make_float2(0.0f, 0.0f);
        constexpr int S = extp(L) / 4;
        const float2 *base = reinterpret_cast<const float2 *>(vbase) + q;
        if constexpr (LOG) {
            constexpr int NQA = (2 * R + 4) / 4 + 1;
            constexpr int NQB = (2 * (R + 1) + 3) / 4 + 1;
            HQuads2<R, tapoff(L), NQA - 1, 1, false, S>::run(base + voff(L) + extp(L), p);
            HQuads2<R + 1, tapoff2(L), NQB - 1, 0, true, S>::run(base + voff(L), p);
        } else {
            constexpr int NQ = (2 * R + 3) / 4 + 1;
            HQuads2<R, tapoff(L), NQ - 1, 0, false, S>::run(base + voff(L), p);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[0][u] = p[u].x;
            a[HR - 1][u] = p[u].y;
        }
    } else if constexpr (HW == 2) {
        float (&a0)[4] = a[0];
        a0[0] = a0[1] = 0.0f;
        if constexpr (LOG) {
            HPairs<R, tapoff(L), (2 * R + 4) / 2 - 1, 1, false>::run(
                reinterpret_cast<const float2 *>(vbase + voff(L) + extp(L)) + q, a0);
            HPairs<R + 1, tapoff2(L), (2 * R + 5) / 2 - 1, 0, true>::run(
                reinterpret_cast<const float2 *>(vbase + voff(L)) + q, a0);
        } else {
            HPairs<R, tapoff(L), (2 * R + 3) / 2 - 1, 0, false>::run(
                reinterpret_cast<const float2 *>(vbase + voff(L)) + q, a0);
        }
    } else {
        float (&a0)[4] = a[0];
#pragma unroll
        for (int u = 0; u < 4; ++u) a0[u] = 0.0f;
        if constexpr (LOG) {
            // t^2 (g (*)_x (g'' (*)_y I) + g'' (*)_x (g (*)_y I)): the first row
            // starts one column before its radius-R window, the second is read
            // with radius R + 1
            constexpr int NQA = (2 * R + 4) / 4 + 1;
            constexpr int NQB = (2 * (R + 1) + 3) / 4 + 1;
            hquads<R, tapoff(L), NQA, 1, false>(
                reinterpret_cast<const float4 *>(vbase + voff(L) + extp(L)) + q, a0);
            hquads<R + 1, tapoff2(L), NQB, 0, true>(
                reinterpret_cast<const float4 *>(vbase + voff(L)) + q, a0);
        } else {
            constexpr int NQ = (2 * R + 3) / 4 + 1;
            hquads<R, tapoff(L), NQ, 0, false>(reinterpret_cast<const float4 *>(vbase + voff(L)) + q,
                                               a0);
        }
    }
}

// The response of level L at one row of the item's outputs from its
// horizontal sums a: the DoG of Eq. 2 with the previous level (kept in
// st.lp), or the scale-normalised Laplacian of the level itself; then the
// running max / argmax, the ring and masks of the 26-neighbour rule, the
// soft-score sums or the stored stack.  `vs` scales the V rows to stretched
// units (1 for the FFMA kernel; the tensor-core kernel keeps the raw MMA
// sums, whose offset drops out of the DoG and the LoG because the taps sum
// to 1 and the second-difference taps to 0).
template <int L>
__device__ __forceinline__ void hrespond(const MhfdKHeader &h, const HCtx &cx, const HRowCtx &w,
                                         HRowState &st, float *soft, const float (&a)[4],
                                         float *s_ring, float vs) {
    if (MODE == 3) {
#pragma unroll
        for (int u = 0; u < HW; ++u)
            if (w.inter[u]) h.stack_out[(long long)w.gy * h.W + cx.gx0 + u] += a[u];
    } else if (!LOG && L == 0) {
#pragma unroll
        for (int u = 0; u < HW; ++u) {
            st.lp[u] = a[u];
            st.m[u] = -__int_as_float(0x7f800000);
            st.a[u] = 0;
            st.mk[u] = 0;
        }
    } else {
        constexpr int I = LOG ? L : (L > 0 ? L - 1 : 0);  // response layer
        constexpr float ts = kTsc(I);                    // t_I, or t_I^2 for the LoG
        const float tsv = ts * vs;
        float d[4];
        if constexpr (LOG) {
#pragma unroll
            for (int u = 0; u < HW; ++u) d[u] = tsv * a[u];
            if (L == 0) {
#pragma unroll
                for (int u = 0; u < HW; ++u) {
                    st.m[u] = -__int_as_float(0x7f800000);
                    st.a[u] = 0;
                    st.mk[u] = 0;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < HW; ++u) {
                d[u] = tsv * (a[u] - st.lp[u]);
                st.lp[u] = a[u];
            }
        }
        if (MODE == 0) {
#pragma unroll
            for (int u = 0; u < HW; ++u)
                if (d[u] > st.m[u]) {
                    st.m[u] = d[u];
                    st.a[u] = I;
                }
        } else if (MODE == 2) {
#pragma unroll
            for (int u = 0; u < HW; ++u)
                if (w.inter[u]) {
                    const float z = fminf(fmaxf((d[u] - h.soft_tau) * h.soft_inv_t, -80.0f), 80.0f);
                    soft[I] += __fdividef(1.0f, 1.0f + __expf(-z));
                }
        } else {
            const float ninf = -__int_as_float(0x7f800000);
            if (mk_ok((unsigned)w.slot < (unsigned)RING)) {
                float *row = s_ring + (w.slot * NDOG + I) * TX2;
                if constexpr (HW == 4)
                    reinterpret_cast<float4 *>(row)[cx.q] =
                        make_float4(w.inb[0] ? d[0] : ninf, w.inb[1] ? d[1] : ninf,
                                    w.inb[2] ? d[2] : ninf, w.inb[3] ? d[3] : ninf);
                else
                    reinterpret_cast<float2 *>(row)[cx.q] =
                        make_float2(w.inb[0] ? d[0] : ninf, w.inb[1] ? d[1] : ninf);
            }
#pragma unroll
            for (int u = 0; u < HW; ++u) {
                if (!w.inb[u]) continue;
                if (I > 0 && d[u] > st.dp[u]) st.mk[u] &= ~(LMask(1) << (I > 0 ? I - 1 : 0));
                if (d[u] > h.thr && (I == 0 || !(st.dp[u] > d[u]))) st.mk[u] |= LMask(1) << I;
                st.dp[u] = d[u];
            }
        }
        if (STORE) {
#pragma unroll
            for (int u = 0; u < HW; ++u)
                if (w.inter[u] && mk_ok((unsigned)w.gy < (unsigned)h.H &&
                                        (unsigned)(cx.gx0 + u) < (unsigned)h.W))
                    h.stack_out[(long long)I * h.plane + (long long)w.gy * h.W + cx.gx0 + u] = d[u];
        }
    }
}

template <int L>
__device__ __forceinline__ void hlevel(const MhfdKHeader &h, const float *vbase, const HCtx &cx,
                                       HState &st, float *s_ring, float vs) {
    float a[HR][4];
    // the item's rows and quad lie in the step (its window columns, fixed at
    // compile time, lie in the level's row of padded width extp(L))
    if (mk_ok(cx.j0 + HR <= RB && (unsigned)cx.q < (unsigned)NQW)) {
        hsums<L>(vbase, cx.q, a);
    } else {
#pragma unroll
        for (int rr = 0; rr < HR; ++rr)
#pragma unroll
            for (int u = 0; u < HW; ++u) a[rr][u] = 0.0f;
    }
#pragma unroll
    for (int rr = 0; rr < HR; ++rr)
        hrespond<L>(h, cx, cx.rw[rr], st.rw[rr], st.soft, a[rr], s_ring, vs);
}

template <int L, int LE>
struct HLevels {
    static __device__ __forceinline__ void run(const MhfdKHeader &h, const float *vbase,
                                               const HCtx &cx, HState &st, float *s_ring,
                                               float vs) {
        hlevel<L>(h, vbase, cx, st, s_ring, vs);
        HLevels<L + 1, LE>::run(h, vbase, cx, st, s_ring, vs);
    }
};
template <int LE>
struct HLevels<LE, LE> {
    static __device__ __forceinline__ void run(const MhfdKHeader &, const float *, const HCtx &,
                                               HState &, float *, float) {}
};

// Chunk geometry: chunk row r is image row yb + r; rows 1..Y are output
// rows, rows 0 and Y + 1 their NMS neighbours.  Output column c of the
// strip (1..TX) is image column x0 - 1 + c.
struct March {
    int x0, yb, Y;
};

__device__ __forceinline__ HCtx make_ctx(const MhfdKHeader &h, const March &m, int item, int s) {
    HCtx cx;
    const int j = item / NQW;
    cx.q = item - j * NQW;
    cx.j0 = HR * j;
    cx.gx0 = m.x0 - 1 + HW * cx.q;
#pragma unroll
    for (int rr = 0; rr < HR; ++rr) {
        HRowCtx &w = cx.rw[rr];
        w.r = s * RB + cx.j0 + rr;
        w.slot = w.r % RING;
        w.gy = m.yb + w.r;
        const bool rowin = w.gy >= 0 && w.gy < h.H;
        const bool rowint = rowin && w.r >= 1 && w.r <= m.Y;
#pragma unroll
        for (int u = 0; u < HW; ++u) {
            const int gx = cx.gx0 + u;
            const int c = HW * cx.q + u;
            w.inb[u] = rowin && gx >= 0 && gx < h.W;
            w.inter[u] = rowint && c >= 1 && c <= TX2 - 2 && gx < h.W;
        }
    }
    return cx;
}

template <int G>
__device__ __forceinline__ void hpass(const MhfdKHeader &h, const March &m, const float *s_v,
                                      float *s_ring, unsigned char *s_arg, HState (&hs)[HI],
                                      int s, float vs = 1.0f) {
#pragma unroll
    for (int it = 0; it < HI; ++it) {
        const int item = threadIdx.x < NTW ? threadIdx.x + it * NTW : HITEMS;
        if (item < HITEMS) {
            const HCtx cx = make_ctx(h, m, item, s);
            const float *vbase = s_v + (HR == 1 ? cx.j0 * VROW : (cx.j0 >> 1) * 2 * VROW);
            HLevels<kGB(G), kGB(G + 1)>::run(h, vbase, cx, hs[it], s_ring, vs);
#pragma unroll
            for (int rr = 0; rr < HR; ++rr) {
                const HRowCtx &w = cx.rw[rr];
                const HRowState &st = hs[it].rw[rr];
                if (!mk_ok((unsigned)w.slot < (unsigned)RING)) continue;
                if (G == NGROUPS - 1 && MODE == 0) {
                    const float ninf = -__int_as_float(0x7f800000);
                    if constexpr (HW == 4) {
                        reinterpret_cast<float4 *>(s_ring + w.slot * TX2)[cx.q] =
                            make_float4(w.inb[0] ? st.m[0] : ninf, w.inb[1] ? st.m[1] : ninf,
                                        w.inb[2] ? st.m[2] : ninf, w.inb[3] ? st.m[3] : ninf);
                        reinterpret_cast<uchar4 *>(s_arg + w.slot * TX2)[cx.q] =
                            make_uchar4((unsigned char)st.a[0], (unsigned char)st.a[1],
                                        (unsigned char)st.a[2], (unsigned char)st.a[3]);
                    } else {
                        reinterpret_cast<float2 *>(s_ring + w.slot * TX2)[cx.q] =
                            make_float2(w.inb[0] ? st.m[0] : ninf, w.inb[1] ? st.m[1] : ninf);
                        reinterpret_cast<uchar2 *>(s_arg + w.slot * TX2)[cx.q] =
                            make_uchar2((unsigned char)st.a[0], (unsigned char)st.a[1]);
                    }
                    if (STORE) {
#pragma unroll
                        for (int u = 0; u < HW; ++u)
                            if (w.inter[u] && mk_ok((unsigned)w.gy < (unsigned)h.H &&
                                                    (unsigned)(cx.gx0 + u) < (unsigned)h.W)) {
                                const long long o2 = (long long)w.gy * h.W + cx.gx0 + u;
                                if (h.m_out) h.m_out[o2] = st.m[u];
                                if (h.arg_out) h.arg_out[o2] = st.a[u];
                            }
                    }
                }
                if (G == NGROUPS - 1 && MODE == 1) {
                    LMask *mrow = reinterpret_cast<LMask *>(s_arg) + w.slot * TX2 + HW * cx.q;
#pragma unroll
                    for (int u = 0; u < HW; ++u) mrow[u] = st.mk[u];
                }
            }
        }
    }
}

template <int G>
struct Groups {
    static __device__ __forceinline__ void run(const MhfdKHeader &h, const March &m,
                                               const float *win, float *s_v, float *s_ring,
                                               unsigned char *s_arg, HState (&hs)[HI], int s) {
        vpass<G>(win, s_v);
        __syncthreads();
        hpass<G>(h, m, s_v, s_ring, s_arg, hs, s);
        __syncthreads();
        Groups<G + 1>::run(h, m, win, s_v, s_ring, s_arg, hs, s);
    }
};
template <>
struct Groups<NGROUPS> {
    static __device__ __forceinline__ void run(const MhfdKHeader &, const March &, const float *,
                                               float *, float *, unsigned char *, HState (&)[HI],
                                               int) {}
};

// ------------------------------------------------------ 4-5. NMS, compaction

// exclusive block scan of one int per thread; *sum receives the total.
// One barrier: the warps' totals go to one of two halves of s_scan
// (alternating with `par`), and every thread adds up the totals itself; the
// barrier of the next scan separates this scan's reads from the writes of
// the scan after it into the same half.
__device__ __forceinline__ int block_excl_scan(int v, int *s_scan, int *sum, int &par) {
    constexpr int NW = NT / 32;
    static_assert(NW <= 32, "two halves of 32 warp totals");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *buf = s_scan + 32 * par;
    par ^= 1;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) buf[warp] = x;
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int t = buf[w];
        before += w < warp ? t : 0;
        total += t;
    }
    *sum = total;
    return before + x - v;
}

// paper rule: M > thr and M >= every 8-neighbour (out-of-image = -inf)
__device__ __forceinline__ bool cand_paper(const float *s_ring, int r, int c, float thr,
                                           float *m_out) {
    const float *row = s_ring + (r % RING) * TX2;
    const float m = row[c];
    *m_out = m;
    if (!(m > thr)) return false;
    const float *up = s_ring + ((r - 1) % RING) * TX2;
    const float *dn = s_ring + ((r + 1) % RING) * TX2;
    const float nb = fmaxf(fmaxf(fmaxf(up[c - 1], up[c]), fmaxf(up[c + 1], row[c - 1])),
                           fmaxf(fmaxf(row[c + 1], dn[c - 1]), fmaxf(dn[c], dn[c + 1])));
    return !(nb > m);
}

// 26-neighbour rule on the response ring, for a layer whose mask bit is set
// (above the threshold, not below its scale neighbours at the same pixel):
// the 8 spatial neighbours of its own layer first, then those of the layers
// below and above (out-of-image neighbours hold -inf)
__device__ __forceinline__ bool cand_26(const float *s_ring, int r, int c, int l, float thr,
                                        float *v_out) {
    const float v = s_ring[((r % RING) * NDOG + l) * TX2 + c];
    *v_out = v;
    if (!(v > thr)) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int ll = l + (k == 0 ? 0 : k == 1 ? -1 : 1);
        if (ll < 0 || ll >= NDOG) continue;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
            const float *row = s_ring + (((r + dr) % RING) * NDOG + ll) * TX2;
            if (row[c - 1] > v || row[c + 1] > v || (dr != 0 && row[c] > v)) return false;
        }
    }
    return true;
}

// Candidates of chunk rows [ra, rb] (all in one tile) appended after `total`
// candidates of that tile's slots; returns the tile's new count.  Items are
// the pixels of the rows in row-major order; under the 26-neighbour rule a
// pixel's layers above the threshold (its mask) are tested in ascending
// order, so candidates come out ordered by row, column, layer.
__device__ __forceinline__ int nms_rows(const MhfdKHeader &h, const March &m,
                                        const float *s_ring, const unsigned char *s_arg,
                                        int *s_scan, int &par, int ra, int rb, long long slot,
                                        int total) {
    const int nrows = rb - ra + 1;
    const int items = nrows * TX;
    // contiguous runs of pixels per thread (candidates come out in row-major
    // order after one scan); an odd run length keeps the lanes' ring reads
    // in distinct banks
    const int ch = ((items + NT - 1) / NT) | 1;
    const int beg = min(items, (int)threadIdx.x * ch);
    const int end = min(items, beg + ch);
    const float thr = h.thr;
    const LMask *s_mask = reinterpret_cast<const LMask *>(s_arg);
    int cnt = 0;
    for (int it = beg; it < end; ++it) {
        const int r = ra + it / TX;
        const int c = 1 + (it - (it / TX) * TX);
        float v;
        if (MODE == 0) {
            cnt += cand_paper(s_ring, r, c, thr, &v) ? 1 : 0;
        } else {
            LMask mk = s_mask[(r % RING) * TX2 + c];
            while (mk) {
                const int l = NDOG > 32 ? __ffsll((long long)mk) - 1 : __ffs((int)mk) - 1;
                mk &= mk - 1;
                cnt += cand_26(s_ring, r, c, l, thr, &v) ? 1 : 0;
            }
        }
    }
    int sum;
    int pos = total + block_excl_scan(cnt, s_scan, &sum, par);
    if (cnt && mk_ok(slot >= 0 && pos >= 0)) {
        MhfdCand *dst = h.stage + slot * h.cap_tile;
        auto put = [&](int r, int c, int l, float v) {
            if (pos < h.cap_tile) {
                MhfdCand cd;
                cd.x = m.x0 - 1 + c;
                cd.y = m.yb + r;
                cd.i = l;
                cd.resp = v;
                dst[pos] = cd;
            }
            ++pos;
        };
        for (int it = beg; it < end; ++it) {
            const int r = ra + it / TX;
            const int c = 1 + (it - (it / TX) * TX);
            float v;
            if (MODE == 0) {
                if (cand_paper(s_ring, r, c, thr, &v)) put(r, c, s_arg[(r % RING) * TX2 + c], v);
            } else {
                LMask mk = s_mask[(r % RING) * TX2 + c];
                while (mk) {
                    const int l = NDOG > 32 ? __ffsll((long long)mk) - 1 : __ffs((int)mk) - 1;
                    mk &= mk - 1;
                    if (cand_26(s_ring, r, c, l, thr, &v)) put(r, c, l, v);
                }
            }
        }
    }
    return total + sum;
}

}  // namespace mk

extern "C" __constant__ int mhfd_smem_bytes = mk::SMEM_BYTES;
extern "C" __constant__ int mhfd_param_bytes = (int)sizeof(mk::KParams);
extern "C" __constant__ int mhfd_ntaps = mk::NTAPS;

namespace mk {

struct Smem {
    float *in, *v, *ring;
    unsigned char *arg;
    int *scan;
    unsigned char *win, *btab, *ctrl;  // tensor-core pass: window, B matrices, mbarriers
};

// Adds this block's sums of every layer (FP64, fixed order) to its slot of
// h.soft_part (zeroed before the launch; only this block writes it).
__device__ __forceinline__ void soft_flush(const MhfdKHeader &h, const HState (&hs)[HI],
                                           int *s_scan) {
    constexpr int NW = NT / 32;
    double *red = reinterpret_cast<double *>(s_scan);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < NSOFT; ++i) {
        double v = 0.0;
#pragma unroll
        for (int it = 0; it < HI; ++it) v += (double)hs[it].soft[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NW; ++w) t += red[w];
            h.soft_part[(long long)blockIdx.x * NSOFT + i] += t;
        }
        __syncthreads();
    }
}

// One march down strip `tx` over its tiles [ta, tb): tile k's candidates go
// to slot slot0 + k * tiles_x + tx.  `sp` carries the image of the job.
__device__ __forceinline__ void march(const MhfdKHeader &h, const MhfdStretch &st, int tiles_x,
                                      int tx, int ta, int tb, long long slot0, const Smem &sm) {
    March m;
    m.x0 = tx * TX;
    m.yb = ta * TY - 1;
    m.Y = min((tb - ta) * TY, h.H - ta * TY);
    Strip sp;
    sp.img = reinterpret_cast<const char *>(h.img);
    sp.pitch = h.pitch;
    sp.H = h.H;
    sp.W = h.W;
    sp.dtype = h.dtype;
    sp.xin = m.x0 - 1 - RMAX;
    sp.yin = m.yb - RMAX;
    const int nsteps = (m.Y + 2 + RB - 1) / RB;

    __syncthreads();  // the previous march's last reads of shared memory
    load_rows(sp, st, sm.in, 0, WIN, 0);
    __syncthreads();

    HState hs[HI];
#pragma unroll
    for (int it = 0; it < HI; ++it)
#pragma unroll
        for (int i = 0; i < NSOFT; ++i) hs[it].soft[i] = 0.0f;
    int base = 0;       // input row held in window row 0
    int tile = 0;       // tile (relative to ta) now receiving candidates
    int total = 0;      // its candidates so far
    int par = 0;        // half of the scan buffer the next block scan uses
#pragma unroll 1
    for (int s = 0; s < nsteps; ++s) {
        const bool more = s + 1 < nsteps;
        Prefetch pf;
        if (more) pf.issue(sp, s * RB + WIN);
        Groups<0>::run(h, m, sm.in + (s * RB - base) * WEXTP, sm.v, sm.ring, sm.arg, hs, s);
        // maxima of the rows whose lower neighbour is now known
        int ra = max(1, s * RB - 1);
        const int rb = min(m.Y, s * RB + RB - 2);
        while ((MODE == 0 || MODE == 1) && ra <= rb) {
            const int tend = min(m.Y, (tile + 1) * TY);  // last row of the tile
            const int re = min(rb, tend);
            total = nms_rows(h, m, sm.ring, sm.arg, sm.scan, par, ra, re,
                             slot0 + (long long)(ta + tile) * tiles_x + tx, total);
            if (re == tend) {
                if (threadIdx.x == 0 && mk_ok(ta + tile < h.tiles_y && tx < tiles_x))
                    h.tile_count[slot0 + (long long)(ta + tile) * tiles_x + tx] = total;
                ++tile;
                total = 0;
            }
            ra = re + 1;
        }
        if (more) {
            // keep the window inside the buffer: the next step reads input
            // rows [(s+1) RB, (s+1) RB + WIN)
            if ((s + 1) * RB + WIN - base > BROWS) {
                shift_window(sm.in, (s + 1) * RB - base, s * RB + WIN - (s + 1) * RB);
                base = (s + 1) * RB;
            }
            pf.store(sp.dtype, st, sm.in, s * RB + WIN - base);
        }
        __syncthreads();
    }
    if constexpr (MODE == 2) soft_flush(h, hs, sm.scan);
}

// Tensor-core march: the vertical pass of each group comes from the MMAs
// issued one step earlier; the rows of step s + 2 are fetched during step s
// and stored at its end, so the MMAs of step s + 1 (issued during step s)
// find their rows in the window.
template <int G>
struct GroupsTC {
    static __device__ __forceinline__ void run(const MhfdKHeader &h, const March &m, TcState &tc,
                                               const TcStretch &ts, const Smem &sm,
                                               HState (&hs)[HI], int s, int nsteps, int base) {
        if constexpr (G < NGROUPS) {
            tc_wait(h, tc, G);
            tc.ph ^= 1u << G;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_read<G>(tc, sm.v, ts);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tc.issuer && s + 1 < nsteps) tc_issue<G>(tc, (s + 1) * RB - base);
            hpass<G>(h, m, sm.v, sm.ring, sm.arg, hs, s, ts.a);
            __syncthreads();
            GroupsTC<G + 1>::run(h, m, tc, ts, sm, hs, s, nsteps, base);
        }
    }
};

template <int G>
__device__ __forceinline__ void tc_issue_all(const TcState &tc, int row0) {
    if constexpr (G < NGROUPS) {
        tc_issue<G>(tc, row0);
        tc_issue_all<G + 1>(tc, row0);
    }
}

__device__ __forceinline__ void tc_wait_all(const MhfdKHeader &h, const TcState &tc) {
    for (int g = 0; g < NGROUPS; ++g) tc_wait(h, tc, g);
}

__device__ __forceinline__ void march_tc(const MhfdKHeader &h, const MhfdStretch &st,
                                         int tiles_x, int tx, int ta, int tb, long long slot0,
                                         const Smem &sm, TcState &tc) {
    March m;
    m.x0 = tx * TX;
    m.yb = ta * TY - 1;
    m.Y = min((tb - ta) * TY, h.H - ta * TY);
    Strip sp;
    sp.img = reinterpret_cast<const char *>(h.img);
    sp.pitch = h.pitch;
    sp.H = h.H;
    sp.W = h.W;
    sp.dtype = h.dtype;
    sp.xin = m.x0 - 1 - RMAX;
    sp.yin = m.yb - RMAX;
    const int nsteps = (m.Y + 2 + RB - 1) / RB;
    const TcStretch ts = tc_stretch(st);

    __syncthreads();  // the previous march's last reads of shared memory
    tc_load_rows(sp, ts, sm.win, 0, WIN + RB);  // the rows of steps 0 and 1
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tc.issuer) tc_issue_all<0>(tc, 0);

    HState hs[HI];
#pragma unroll
    for (int it = 0; it < HI; ++it)
#pragma unroll
        for (int i = 0; i < NSOFT; ++i) hs[it].soft[i] = 0.0f;
    int base = 0;       // input row held in window row 0
    int tile = 0;       // tile (relative to ta) now receiving candidates
    int total = 0;      // its candidates so far
    int par = 0;        // half of the scan buffer the next block scan uses
#pragma unroll 1
    for (int s = 0; s < nsteps; ++s) {
        const bool more2 = s + 2 < nsteps;
        Prefetch pf;
        if (more2) pf.issue(sp, (s + 1) * RB + WIN);  // the new rows of step s + 2
        GroupsTC<0>::run(h, m, tc, ts, sm, hs, s, nsteps, base);
        int ra = max(1, s * RB - 1);
        const int rb = min(m.Y, s * RB + RB - 2);
        while (ra <= rb) {
            const int tend = min(m.Y, (tile + 1) * TY);
            const int re = min(rb, tend);
            total = nms_rows(h, m, sm.ring, sm.arg, sm.scan, par, ra, re,
                             slot0 + (long long)(ta + tile) * tiles_x + tx, total);
            if (re == tend) {
                if (threadIdx.x == 0 && mk_ok(ta + tile < h.tiles_y && tx < tiles_x))
                    h.tile_count[slot0 + (long long)(ta + tile) * tiles_x + tx] = total;
                ++tile;
                total = 0;
            }
            ra = re + 1;
        }
        if (more2) {
            // the window must hold rows [(s+1) RB, (s+2) RB + WIN) and the
            // 16 rows past them that padded K ranges read
            if ((s + 2) * RB + WIN + 16 - base > BROWS) {
                tc_wait_all(h, tc);  // the MMAs of step s + 1 read the window
                tc_shift(sm.win, (s + 1) * RB - base, WIN);
                base = (s + 1) * RB;
                __syncthreads();
            }
            tc_store_prefetch(pf, ts, sm.win, (s + 1) * RB + WIN - base);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        // no barrier here: the rows just stored are first read by MMAs issued
        // after the next step's first readout barrier; the V rows, the ring
        // and the scan buffer are each guarded by an earlier barrier (the
        // last group's, and the next scan's)
    }
}

#if MHFD_VTC == 2
// ------------------------------------------------- two-pass kernel (TC2)
//
// Both separable blur passes are tensor-core products, on tiles of T2M = 128
// computed rows (the TY output rows and their two NMS neighbours) by TX2
// computed columns.  The window X holds the tile's input rows and columns
// with a halo of RMAX on every side as exact fp16 integers x = clamp(v, lo,
// hi) - c0 (MN-major: column group cg of 8 columns at cg * T2_XGSTR, row r at
// + 16 r).  Per level l (all levels of §2.2's ladder, in order):
//   vertical    V_l[m, c'] = sum_k G_l[m, k] X[k0 + k, j0 + c']: A = the
//               level's banded tap matrix (taps g_l[|k - m - R_l|] scaled by
//               T2_S and split into fp16 hi + lo parts), M = 128 rows in
//               reverse order, K-major; B = the window, MN-major; N = the V
//               columns; f32 accumulators in tensor memory;
//   split       the f32 V_l into fp16 hi + lo parts (hi: V with its low 13
//               mantissa bits cleared, exact in fp16; lo = V - hi), written
//               as rows m by columns k = c' - off (K-major) to shared memory;
//   horizontal  L_l[m, c] = sum_k V_l[m, k] T_l[k, c], T_l[k, c] = g_l[|k - c -
//               R_l|]: A = the split rows, B = the same banded tap matrix,
//               N = TX2 computed columns in reverse order; the products hi x
//               hi, hi x lo and lo x hi;
//   epilogue    D_{l-1} = t_{l-1} (L_l - L_{l-1}) (Eq. 2) and the running max
//               over scales with its first argmax (Eq. 3), per pixel in
//               registers.
// A banded tap matrix is Toeplitz: with the M (or N) index reversed, an 8 x 8
// block of it depends only on the sum of its block row and column, so one
// column of T2_SMAX blocks, addressed with equal leading and stride offsets
// (128 bytes), serves every M tile and K step of both products.
// The last warp issues the MMAs (one elected lane of a converged warp: the
// descriptors stay warp-uniform); the other 8 warps (workers) split, build
// the tap matrices of the level after next, form the responses and run the
// NMS and compaction of the tile.  Handoffs go through mbarriers:
//   VB[b] / HB[b]  vertical / horizontal products of a level done (commit),
//   SPL            a level's split done (8 worker warps),
//   XR             the next tile's window and first two tap matrices ready.
// Level l of the block's g-th level overall uses V buffer (g mod 2), L buffer
// (g mod 2) and tap-matrix buffer (g mod 3): the tensor core runs level l's
// horizontal product and level l + 2's vertical one while the workers split
// level l + 1, so every buffer is free when it is written.  All waits are
// bounded (2 s of global time); a wait that gives up sets h.flag and makes
// every later wait of the block return at once.

constexpr float T2_S = 16.0f;  // tap scale: |V| <= 2048 * 16 fits fp16

// Per-level constants, read at run time from constant memory: the level
// loop is not unrolled (17 unrolled levels overflowed the instruction cache).
struct T2Lev {
    int r, kv16, nv, kh16, off, need, j0, k0, s, toff;
    float tsc;  // t of the response layer this level closes (level - 1)
};
struct T2Levs {
    T2Lev v[NL];
};
MK_HD constexpr T2Levs t2_levs() {
    T2Levs t{};
    for (int l = 0; l < NL; ++l)
        t.v[l] = T2Lev{kR(l),       t2_kv(l) / 16, t2_nv(l), t2_kh(l) / 16, t2_off(l), t2_need(l),
                       t2_j0(l),    t2_k0(l),      t2_s(l),  tapoff(l),     l > 0 ? kTsc(l - 1) : 0.0f};
    return t;
}
__constant__ T2Levs mk_t2_levs = t2_levs();
MK_HD constexpr int t2_kv16max() {
    int m = 0;
    for (int l = 0; l < NL; ++l) m = t2_kv(l) / 16 > m ? t2_kv(l) / 16 : m;
    return m;
}
constexpr int T2_CP = (T2_NW / 32) / 4;  // column parts: worker warps per tensor-memory lane group
constexpr int T2_CQ = TX2 / T2_CP;       // L columns of a worker thread

// the block's dynamic shared memory (the same array as the kernel's)
extern __shared__ __align__(16) unsigned char mk_t2_smem[];
struct T2State {
    unsigned tmem;      // tensor-memory base (lane 0, column 0)
    unsigned ph;        // mbarrier parities: VB0 VB1 HB0 HB1 (workers), SPL XR (issuer)
    unsigned g;         // levels run by this block so far
    // shared-memory regions: window, tap matrices, split rows, control block
    __device__ __forceinline__ unsigned char *xp() const { return mk_t2_smem; }
    __device__ __forceinline__ unsigned char *tabp() const { return mk_t2_smem + T2_OFF_TAB; }
    __device__ __forceinline__ unsigned char *ahp() const { return mk_t2_smem + T2_OFF_AH; }
    __device__ __forceinline__ unsigned char *ctrl() const { return mk_t2_smem + T2_OFF_CTRL; }
    __device__ __forceinline__ unsigned x() const { return smem_addr(xp()); }
    __device__ __forceinline__ unsigned tab() const { return smem_addr(tabp()); }
    __device__ __forceinline__ unsigned ah() const { return smem_addr(ahp()); }
    __device__ __forceinline__ int *scan() const { return reinterpret_cast<int *>(ctrl() + 128); }
    __device__ __forceinline__ int *cmap() const { return reinterpret_cast<int *>(ctrl() + 512); }
    // 26-neighbour rule: exchange buffer b, kept-layer masks
    __device__ __forceinline__ float *l26x(int b) const {
        return reinterpret_cast<float *>(mk_t2_smem + T2_OFF_L26 + b * T2_L26_XB);
    }
    __device__ __forceinline__ unsigned short *l26m() const {
        return reinterpret_cast<unsigned short *>(mk_t2_smem + T2_OFF_L26 + 2 * T2_L26_XB);
    }
    __device__ __forceinline__ volatile int *fail() const {
        return reinterpret_cast<volatile int *>(ctrl() + 100);
    }
};
__device__ __forceinline__ unsigned t2_bar(const T2State &t, int i) { return smem_addr(t.ctrl()) + 8u * i; }
// mbarriers: VB0 VB1 HB0 HB1 (product commits), SPL and XR (worker warps),
// TB0..TB3 (tap-matrix copies into buffer 0..3)
enum { T2_VB = 0, T2_HB = 2, T2_SPL = 4, T2_XRB = 5, T2_TB = 6 };

__device__ __forceinline__ void t2_wait(const MhfdKHeader &h, T2State &t, int i) {
    const unsigned bar = t2_bar(t, i), par = (t.ph >> i) & 1u;
    t.ph ^= 1u << i;
    if (tc_try(bar, par) || *t.fail()) return;
    const unsigned long long t0 = gtimer();
    for (;;) {
#pragma unroll 1
        for (int k = 0; k < 256; ++k)
            if (tc_try(bar, par)) return;
        if (*t.fail()) return;
        if (gtimer() - t0 > 2000000000ull) break;
    }
    *t.fail() = 1;
    if (h.flag) atomicOr(h.flag, 1);
}

__device__ __forceinline__ void t2_mma(unsigned d, unsigned long long a, unsigned long long b,
                                       unsigned idesc, unsigned acc) {
    asm volatile(
        "{\n.reg .pred q, e;\nsetp.ne.b32 q, %4, 0;\nelect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// the same with the descriptors formed inside the statement (base + constant
// offsets): unrolled K loops then keep only the two bases in registers
template <unsigned long long OA, unsigned long long OB, unsigned ACC>
__device__ __forceinline__ void t2_mma_o(unsigned d, unsigned long long a0, unsigned long long b0,
                                         unsigned idesc) {
    asm volatile(
        "{\n.reg .pred q, e;\n.reg .b64 a, b;\nadd.u64 a, %1, %4;\nadd.u64 b, %2, %5;\n"
        "setp.ne.b32 q, %6, 0;\nelect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, q;\n}\n" ::"r"(d),
        "l"(a0), "l"(b0), "r"(idesc), "n"(OA), "n"(OB), "n"(ACC)
        : "memory");
}
// K steps KK .. NKMAX - 1 of a product, those below nk issued (a warp-uniform
// branch per step; the offsets stay compile-time constants)
template <int KK, int NKMAX>
struct T2VK {  // vertical: (hi, window), (lo, window)
    static __device__ __forceinline__ void run(unsigned d, unsigned long long a0, unsigned long long b0,
                                               unsigned id, int nk) {
        if constexpr (KK < NKMAX) {
            if (KK < nk) {
                t2_mma_o<(unsigned long long)(KK * 16), (unsigned long long)(KK * 16), KK ? 1u : 0u>(d, a0, b0,
                                                                                                   id);
                t2_mma_o<(unsigned long long)(KK * 16 + (T2_TAB_PART >> 4)), (unsigned long long)(KK * 16),
                         1u>(d, a0, b0, id);
                T2VK<KK + 1, NKMAX>::run(d, a0, b0, id, nk);
            }
        }
    }
};
template <int KK, int NKMAX>
struct T2HK {  // horizontal: hi x hi, hi x lo, lo x hi
    static __device__ __forceinline__ void run(unsigned d, unsigned long long a0, unsigned long long b0,
                                               unsigned id, int nk) {
        if constexpr (KK < NKMAX) {
            if (KK < nk) {
                t2_mma_o<(unsigned long long)(KK * 16), (unsigned long long)(KK * 16), KK ? 1u : 0u>(d, a0, b0,
                                                                                                   id);
                t2_mma_o<(unsigned long long)(KK * 16), (unsigned long long)(KK * 16 + (T2_TAB_PART >> 4)),
                         1u>(d, a0, b0, id);
                t2_mma_o<(unsigned long long)(KK * 16 + (T2_AH_PART >> 4)), (unsigned long long)(KK * 16),
                         1u>(d, a0, b0, id);
                T2HK<KK + 1, NKMAX>::run(d, a0, b0, id, nk);
            }
        }
    }
};
__device__ __forceinline__ void t2_commit(unsigned bar) {
    asm volatile(
        "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
        : "memory");
}
// one arrival per worker warp, after every lane's shared-memory writes (made
// visible to the tensor core) and tensor-memory reads
__device__ __forceinline__ void t2_arrive(unsigned bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if ((threadIdx.x & 31) == 0)
        asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar)
                     : "memory");
}
__device__ __forceinline__ void t2_wsync() { asm volatile("bar.sync 1, %0;" ::"n"(T2_NW) : "memory"); }

__device__ __forceinline__ unsigned t2_tabb(const T2State &t, unsigned gl) {
    return t.tab() + (gl % (unsigned)T2_NTAB) * (unsigned)(2 * T2_TAB_PART);
}
// Copy level l's tap matrices (built once per detector in global memory by
// mhfd_t2_tables) into buffer gl mod T2_NTAB with the bulk-copy engine; the
// buffer's mbarrier completes when the bytes have landed.
__device__ __forceinline__ void t2_fetch_tab(const MhfdKHeader &h, const T2State &t, int l, unsigned gl) {
    const unsigned b = gl % (unsigned)T2_NTAB;
    const unsigned bar = t2_bar(t, T2_TB + (int)b);
    const unsigned dst = t2_tabb(t, gl);
    const char *src = reinterpret_cast<const char *>(h.t2tab) + (long long)l * (2 * T2_TAB_PART);
    asm volatile(
        "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
        "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
        "@e cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %1, [%0];\n}\n" ::"r"(bar),
        "n"(2 * T2_TAB_PART), "r"(dst), "l"(src)
        : "memory");
}

// vertical product of level l into V buffer column dcol
__device__ __forceinline__ void t2_issue_v(const T2State &t, int l, unsigned tabb, unsigned dcol) {
    const T2Lev &lv = mk_t2_levs.v[l];
    const unsigned id =
        (1u << 4) | (1u << 16) | ((unsigned)(lv.nv >> 3) << 17) | ((unsigned)(T2M >> 4) << 24);
    const unsigned long long a0 = tc_desc(tabb, 128u, 128u);
    const unsigned long long b0 =
        tc_desc(t.x() + (unsigned)((lv.j0 / 8) * T2_XGSTR + lv.k0 * 16), 128u, (unsigned)T2_XGSTR);
    // unrolled with constant descriptor offsets: the issue keeps the tensor
    // core's pace (a rolled loop issued one MMA per ~70 cycles on GB300)
    T2VK<0, t2_kv16max()>::run(t.tmem + dcol, a0, b0, id, lv.kv16);
}
// horizontal product of level l into L buffer column dcol
__device__ __forceinline__ void t2_issue_h(const T2State &t, int l, unsigned tabb, unsigned dcol) {
    constexpr unsigned ID = (1u << 4) | ((unsigned)(TX2 >> 3) << 17) | ((unsigned)(T2M >> 4) << 24);
    constexpr int BOFF = 16 - TX2 / 8;  // reversed N: block row + column - BOFF = 15 at the diagonal
    const unsigned long long a0 = tc_desc(t.ah(), 128u, (unsigned)T2_SBO_H);
    const unsigned long long b0 = tc_desc(tabb + BOFF * 128, 128u, 128u);
    T2HK<0, T2_KHMAX / 16>::run(t.tmem + dcol, a0, b0, ID, mk_t2_levs.v[l].kh16);
}

// The banded tap matrix of level l: block s, row a, column b holds
// g_l[|8 s + a + b - 127 - R_l|] * T2_S (0 beyond R_l), hi part then lo part.
__device__ __forceinline__ void t2_build_tab(unsigned char *tab, int l, int wt) {
    const T2Lev &lv = mk_t2_levs.v[l];
    const int R = lv.r, S = lv.s, toff = lv.toff;
#pragma unroll 1
    for (int it = wt; it < S * 8; it += T2_NW) {
        const int s = it >> 3, a = it & 7;
        unsigned hi[4], lo[4];
#pragma unroll
        for (int b = 0; b < 8; b += 2) {
            unsigned short h2[2], l2[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                int d = 8 * s + a + b + e - 127 - R;
                d = d < 0 ? -d : d;
                const float v = d <= R ? mk_taps_rt[toff + d] * T2_S : 0.0f;
                h2[e] = f2h_rn(v);
                l2[e] = f2h_rn(v - h2f(h2[e]));
            }
            hi[b >> 1] = (unsigned)h2[0] | ((unsigned)h2[1] << 16);
            lo[b >> 1] = (unsigned)l2[0] | ((unsigned)l2[1] << 16);
        }
        if (mk_ok(s < T2_SMAX)) {
            *reinterpret_cast<uint4 *>(tab + s * 128 + a * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(tab + T2_TAB_PART + s * 128 + a * 16) =
                make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

__device__ __forceinline__ unsigned t2_pack(float lo_half, float hi_half) {
    unsigned r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_half), "f"(lo_half));
    return r;
}

// Split of level l: V buffer column dcol (tensor memory, lane = row) into the
// hi and lo rows of the horizontal product's A operand.  Worker warp w takes
// lanes 32 (w mod 4) .. + 31 and part w / 4 of the 8-column blocks.  OFF
// (the level's V column of A column 0) selects registers, so it is a
// template parameter; t2_split dispatches on it.
template <int OFF>
__device__ __forceinline__ void t2_split_o(const T2State &t, unsigned dcol, int kb, int need, int wt) {
    const int w = wt >> 5, g = w & 3, q = w >> 2;
    const int row = 32 * g + (wt & 31);
    const unsigned taddr = t.tmem + ((unsigned)(32 * g) << 16) + dcol;
    unsigned char *dst = t.ahp() + (row >> 3) * T2_SBO_H + (row & 7) * 16;
    const int jb = q * kb / T2_CP, je = (q + 1) * kb / T2_CP;
#pragma unroll 1
    for (int j = jb; j < je; ++j) {
        unsigned r0[8], r1[8];
        tc_ld8(taddr + (unsigned)(8 * j), r0);
        if constexpr (OFF != 0) tc_ld8(taddr + (unsigned)(8 * j + 8), r1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 8; e += 4) {
            asm volatile("" : "+r"(r0[e]), "+r"(r0[e + 1]), "+r"(r0[e + 2]), "+r"(r0[e + 3]));
            if constexpr (OFF != 0)
                asm volatile("" : "+r"(r1[e]), "+r"(r1[e + 1]), "+r"(r1[e + 2]), "+r"(r1[e + 3]));
        }
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(OFF + e < 8 ? r0[OFF + e] : r1[(OFF + e) & 7]);
        if (8 * j + 8 > need) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (8 * j + e >= need) v[e] = 0.0f;
        }
        unsigned hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const float h0 = __uint_as_float(__float_as_uint(v[e]) & 0xFFFFE000u);
            const float h1 = __uint_as_float(__float_as_uint(v[e + 1]) & 0xFFFFE000u);
            hi[e >> 1] = t2_pack(h0, h1);
            // v - hi, two at a time (exact: the remainder fits f32)
            const float2 l2 = __ffma2_rn(make_float2(h0, h1), make_float2(-1.0f, -1.0f),
                                         make_float2(v[e], v[e + 1]));
            lo[e >> 1] = t2_pack(l2.x, l2.y);
        }
        if (mk_ok(j < T2_KHMAX / 8 && row < T2M)) {
            *reinterpret_cast<uint4 *>(dst + j * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(dst + T2_AH_PART + j * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}
__device__ __forceinline__ void t2_split(const T2State &t, int l, unsigned dcol, int wt) {
    const T2Lev &lv = mk_t2_levs.v[l];
    const int kb = 2 * lv.kh16, need = lv.need;
    switch (lv.off) {
        case 0: t2_split_o<0>(t, dcol, kb, need, wt); break;
        case 1: t2_split_o<1>(t, dcol, kb, need, wt); break;
        case 2: t2_split_o<2>(t, dcol, kb, need, wt); break;
        case 3: t2_split_o<3>(t, dcol, kb, need, wt); break;
        case 4: t2_split_o<4>(t, dcol, kb, need, wt); break;
        case 5: t2_split_o<5>(t, dcol, kb, need, wt); break;
        case 6: t2_split_o<6>(t, dcol, kb, need, wt); break;
        default: t2_split_o<7>(t, dcol, kb, need, wt); break;
    }
}

// per-thread state of the responses: T2_CQ computed columns of one row
struct T2Px {
    float mx[T2_CQ];          // paper rule: running max over scales;
                              // 26-neighbour rule: the previous layer's 3x3 maxima
    unsigned ag[T2_CQ / 4];   // paper rule: first argmax, one byte per column
    // 26-neighbour rule, one bit per column: items of the previous layer
    // waiting for the layer above, columns with a kept item in this tile,
    // pixels inside the image, output pixels
    unsigned fl, any, ci, cv;
};
__device__ __forceinline__ int t2_ag(const T2Px &px, int u) { return (px.ag[u >> 2] >> (8 * (u & 3))) & 0xFF; }
struct T2Tile {
    int oy, ox;   // first output row / column of the tile
};

// Epilogue of level l: L buffer column dcol into the responses.  The
// thread's row is lane 32 (w mod 4) + lane (computed row 127 - that), its
// columns part w / 4 of the reversed columns.
__device__ __forceinline__ void t2_epi(const MhfdKHeader &h, const T2State &t, int l, unsigned dcol, int wt,
                                       T2Px &px, float sc, const T2Tile &tl) {
    const int w = wt >> 5, g = w & 3, q = w >> 2;
    const unsigned taddr = t.tmem + ((unsigned)(32 * g) << 16) + dcol + (unsigned)(T2_CQ * q);
    // the previous level's L: a copy in tensor memory (column T2_LP + the
    // same offset), replaced by this level's
    const unsigned paddr = t.tmem + ((unsigned)(32 * g) << 16) + (unsigned)(T2_LP + T2_CQ * q);
    const bool first = l == 0, last = l + 1 == NL;
    const int I = l - 1;
    const float ts = mk_t2_levs.v[l].tsc * sc;
    constexpr int EC = 4;  // columns per load round
    static_assert(T2_CQ % EC == 0, "whole load rounds");
#pragma unroll
    for (int i0 = 0; i0 < T2_CQ; i0 += EC) {
        unsigned r[EC], rp[EC];
        tc_ld4(taddr + (unsigned)i0, r);
        tc_ld4(paddr + (unsigned)i0, rp);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < EC; e += 4) {
            asm volatile("" : "+r"(r[e]), "+r"(r[e + 1]), "+r"(r[e + 2]), "+r"(r[e + 3]));
            asm volatile("" : "+r"(rp[e]), "+r"(rp[e + 1]), "+r"(rp[e + 2]), "+r"(rp[e + 3]));
        }
        if (!last) {
#pragma unroll
            for (int e = 0; e < EC; e += 4)
                asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                 paddr + (unsigned)(i0 + e)),
                             "r"(r[e]), "r"(r[e + 1]), "r"(r[e + 2]), "r"(r[e + 3])
                             : "memory");
        }
        if (first) {
#pragma unroll
            for (int e = 0; e < EC; ++e) px.mx[i0 + e] = -__int_as_float(0x7f800000);
#pragma unroll
            for (int e = 0; e < EC; e += 4) px.ag[(i0 + e) >> 2] = 0;
        } else {
            // the DoG two columns at a time: (L_l - L_{l-1}) rounded once,
            // then the scale, as the scalar form rounds them
            float dd[EC];
#pragma unroll
            for (int e = 0; e < EC; e += 2) {
                const float2 df = __fmul2_rn(
                    make_float2(ts, ts),
                    __ffma2_rn(make_float2(__uint_as_float(rp[e]), __uint_as_float(rp[e + 1])),
                               make_float2(-1.0f, -1.0f),
                               make_float2(__uint_as_float(r[e]), __uint_as_float(r[e + 1]))));
                dd[e] = df.x;
                dd[e + 1] = df.y;
            }
#pragma unroll
            for (int e = 0; e < EC; ++e) {
                const int u = i0 + e;
                const float d = dd[e];
                if (d > px.mx[u]) {
                    px.mx[u] = d;
                    px.ag[u >> 2] = (px.ag[u >> 2] & ~(0xFFu << (8 * (u & 3)))) | ((unsigned)I << (8 * (u & 3)));
                }
                if (STORE) {
                    const int m = T2M - 1 - (32 * g + (wt & 31));
                    const int c = TX2 - 1 - (T2_CQ * q + u);
                    const int gy = tl.oy - 1 + m, gx = tl.ox - 1 + c;
                    if (m >= 1 && m <= T2M - 2 && c >= 1 && c <= TX2 - 2 && gy < h.H && gx < h.W &&
                        mk_ok(gy >= 0 && gx >= 0))
                        h.stack_out[(long long)I * h.plane + (long long)gy * h.W + gx] = d;
                }
            }
        }
    }
    if (!last) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 26-neighbour rule (the 3x3x3 test of §3 on the layers of Eq. 2), one layer
// at a time, in the epilogue of level l (layer I = l - 1).  With S_I the 3x3
// maximum of D_I around a pixel (neighbours outside the image compare as
// -inf), an item (pixel, I) is kept when D_I > thr, D_I is not below any of
// its 8 neighbours in layer I (so D_I = S_I there), and not below S_{I-1} or
// S_{I+1}.  So once D_I is formed: an item of layer I - 1 flagged one level
// earlier is kept if its response (px.mx, which is S_{I-1} there) is not
// below S_I; the items of layer I that pass the first three tests are
// flagged to wait for the layer above (the top layer keeps them at once);
// px.mx becomes S_I.  D_I replaces L_l in its tensor-memory buffer (free
// until level l + 2's horizontal product, issued after the workers' next
// split) and is read back a round at a time for the test.  The 3x3 maxima
// take the rows above and below from the neighbouring lanes (warp
// shuffles), the segment ends and the lane-group boundary rows from an
// exchange buffer in shared memory (two, alternating by layer: one barrier
// per layer).  A kept item sets bit I of its pixel's mask in shared memory
// and stores its response in the block's scratch, both read at the tile end.
__device__ __forceinline__ void t2_epi26(const MhfdKHeader &h, const T2State &t, int l, unsigned dcol,
                                         T2Px &px, float sc, const T2Tile &tl) {
    constexpr int CQ = T2_CQ, CP = T2_CP;
    const float ninf = -__int_as_float(0x7f800000);
    // the worker thread's index read afresh (volatile): what derives from it
    // is not hoisted out of the level loop, where it would hold registers
    // through the split and the window load
    int wt;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(wt));
    const int w = wt >> 5, lane = wt & 31, g = w & 3, q = w >> 2;
    const int mr = 32 * g + lane, m = T2M - 1 - mr;
    const unsigned taddr = t.tmem + ((unsigned)(32 * g) << 16) + dcol + (unsigned)(CQ * q);
    const unsigned paddr = t.tmem + ((unsigned)(32 * g) << 16) + (unsigned)(T2_LP + CQ * q);
    const bool first = l == 0, last = l + 1 == NL;
    const int I = l - 1;
    const float ts = mk_t2_levs.v[l].tsc * sc;
    if (first) {
        // the tile's pixels inside the image, and its output pixels
        const int gy = tl.oy - 1 + m;
        const bool rowin = gy >= 0 && gy < h.H, rowint = rowin && m >= 1 && m <= T2M - 2;
        unsigned ci = 0, cv = 0;
#pragma unroll
        for (int u = 0; u < CQ; ++u) {
            const int c = TX2 - 1 - (CQ * q + u), gx = tl.ox - 1 + c;
            const bool in = rowin && gx >= 0 && gx < h.W;
            ci |= (unsigned)in << u;
            cv |= (unsigned)(in && rowint && c >= 1 && c <= TX2 - 2) << u;
        }
        px.ci = ci;
        px.cv = cv;
        px.fl = 0;
        px.any = 0;
    }
    float *xc = t.l26x(I & 1);      // [CP parts][2 ends][T2M lanes]
    float *xr = xc + T2M * CP * 2;  // [4 lane groups][2 ends][CP parts][CQ + 4]
    constexpr int XRS = CQ + 4;
    float d0 = 0.0f, dl = 0.0f;     // the segment's ends
    constexpr int EC = 4;
    static_assert(CQ % EC == 0, "whole load rounds");
#pragma unroll
    for (int i0 = 0; i0 < CQ; i0 += EC) {
        unsigned r[EC], rp[EC];
        tc_ld4(taddr + (unsigned)i0, r);
        tc_ld4(paddr + (unsigned)i0, rp);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
        asm volatile("" : "+r"(rp[0]), "+r"(rp[1]), "+r"(rp[2]), "+r"(rp[3]));
        if (!last)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                             paddr + (unsigned)i0),
                         "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3])
                         : "memory");
        if (!first) {
            float dv[EC], dd[EC];
#pragma unroll
            for (int e = 0; e < EC; e += 2) {
                const float2 df = __fmul2_rn(
                    make_float2(ts, ts),
                    __ffma2_rn(make_float2(__uint_as_float(rp[e]), __uint_as_float(rp[e + 1])),
                               make_float2(-1.0f, -1.0f),
                               make_float2(__uint_as_float(r[e]), __uint_as_float(r[e + 1]))));
                dd[e] = df.x;
                dd[e + 1] = df.y;
            }
#pragma unroll
            for (int e = 0; e < EC; ++e) {
                const int u = i0 + e;
                const float v = dd[e];
                if (STORE) {
                    const int c = TX2 - 1 - (CQ * q + u);
                    const int gy = tl.oy - 1 + m, gx = tl.ox - 1 + c;
                    if ((px.cv >> u) & 1u)
                        h.stack_out[(long long)I * h.plane + (long long)gy * h.W + gx] = v;
                }
                dv[e] = (px.ci >> u) & 1u ? v : ninf;
            }
            asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                             taddr + (unsigned)i0),
                         "f"(dv[0]), "f"(dv[1]), "f"(dv[2]), "f"(dv[3])
                         : "memory");
            if (i0 == 0) d0 = dv[0];
            if (i0 + EC == CQ) dl = dv[EC - 1];
            // the whole rows of lanes 0 and 31
            if (lane == 0 || lane == 31)
                *reinterpret_cast<float4 *>(xr + ((g * 2 + (lane == 31 ? 1 : 0)) * CP + q) * XRS + i0) =
                    make_float4(dv[0], dv[1], dv[2], dv[3]);
        }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    if (first) {
        // no layer below the first
#pragma unroll
        for (int u = 0; u < CQ; ++u) px.mx[u] = ninf;
        return;
    }
    if (mk_ok(mr < T2M && q < CP)) {
        xc[(q * 2 + 0) * T2M + mr] = d0;
        xc[(q * 2 + 1) * T2M + mr] = dl;
    }
    t2_wsync();
    // the neighbour row of lane 0 (above) or 31 (below) in the next lane
    // group; none past the tile
    const float *rx = lane == 0 && g > 0    ? xr + (((g - 1) * 2 + 1) * CP + q) * XRS
                      : lane == 31 && g < 3 ? xr + (((g + 1) * 2 + 0) * CP + q) * XRS
                                            : nullptr;
    const unsigned rxh = rx != nullptr, rxa = rx ? smem_addr(rx) : 0u;
    // column max of the three rows just outside the segment (other part)
    auto edge = [&](int qq, int e) {
        if (qq < 0 || qq >= CP) return ninf;
        const float *c = xc + (qq * 2 + e) * T2M;
        float v = c[mr];
        if (mr > 0) v = fmaxf(v, c[mr - 1]);
        if (mr < T2M - 1) v = fmaxf(v, c[mr + 1]);
        return v;
    };
    // D > thr as D >= the next float up, so that the threshold joins the
    // maxima the response must reach
    const float thrp = nextafterf(h.thr, __int_as_float(0x7f800000));
    const bool top = I + 2 == NL;  // the last layer: no layer above
    // the block's scratch: [layer][column u][worker thread]
    constexpr int LAY = CQ * T2_NW;
    const int gvc = ((int)blockIdx.x * (NL - 1) + I) * LAY + wt;
    unsigned ge = 0, nf = 0;
    // pixel uu: its 8 neighbours are the column maxima (three rows) at uu - 1
    // and uu + 1 and the rows above and below at uu (ud, which may also hold
    // the pixel itself).  ge: not below S_I (for an item flagged one layer
    // down, whose response is px.mx); nf: above the threshold and not below
    // its 8 neighbours or S_{I-1} (its response to the scratch at once)
    auto test = [&](int uu, float x, float cl, float cr, float ud) {
        const float nb = fmaxf(fmaxf(cl, cr), ud);
        const float s = fmaxf(nb, x);
        if (!(s > px.mx[uu])) ge |= 1u << uu;
        if (!(fmaxf(fmaxf(nb, px.mx[uu]), thrp) > x)) {
            nf |= 1u << uu;
            h.l26val[gvc + uu * T2_NW] = x;
        }
        px.mx[uu] = s;
    };
    float cprev = edge(q - 1, 1);  // column max at u - 2 (n' = CQ q - 1 at first)
    float ccur = 0.0f, vcur = 0.0f, xcur = 0.0f;  // at u - 1: column max, rows above and below, D
#pragma unroll
    for (int i0 = 0; i0 < CQ; i0 += 4) {
        unsigned r[4];
        tc_ld4(taddr + (unsigned)i0, r);
        // this round's columns of the other lane group's row (lanes 0 and
        // 31: the row above or below; -inf elsewhere)
        float ev[4] = {ninf, ninf, ninf, ninf};
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %5, 0;\n@p ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n}\n"
            : "+f"(ev[0]), "+f"(ev[1]), "+f"(ev[2]), "+f"(ev[3])
            : "r"(rxa + 4u * (unsigned)i0), "r"(rxh)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int u = i0 + e;
            const float x = __uint_as_float(r[e]);
            // rows above and below: lanes 0 and 31 get their own value from
            // the shuffles, which leaves the tests unchanged (a pixel is not
            // below itself); volatile: the shuffles stay in column order, so
            // that they do not all occupy registers at once
            float up, dn;
            asm volatile("shfl.sync.up.b32 %0, %1, 1, 0, 0xffffffff;" : "=f"(up) : "f"(x));
            asm volatile("shfl.sync.down.b32 %0, %1, 1, 31, 0xffffffff;" : "=f"(dn) : "f"(x));
            const float vn = fmaxf(fmaxf(up, dn), ev[e]), cn = fmaxf(vn, x);
            if (u > 0) {
                test(u - 1, xcur, cprev, cn, vcur);
                cprev = ccur;
            }
            xcur = x;
            vcur = vn;
            ccur = cn;
        }
    }
    test(CQ - 1, xcur, cprev, edge(q + 1, 0), vcur);  // n' = CQ q + CQ past the segment
    // kept: the flagged items of layer I - 1 not below S_I; flags only on
    // output pixels
    const unsigned fin = px.fl & ge;
    nf &= px.cv;
    px.fl = top ? 0u : nf;
    unsigned short *msk = t.l26m() + wt;  // [column u][worker thread]
#pragma unroll 1
    for (unsigned f = fin; f; f &= f - 1) {
        const int uu = __ffs(f) - 1;
        if (mk_ok(uu < CQ && wt < T2_NW))
            msk[uu * T2_NW] = (unsigned short)(msk[uu * T2_NW] | (1u << (I - 1)));
    }
    if (top) {
#pragma unroll 1
        for (unsigned f = nf; f; f &= f - 1) {
            const int uu = __ffs(f) - 1;
            if (mk_ok(uu < CQ && wt < T2_NW)) msk[uu * T2_NW] = (unsigned short)(msk[uu * T2_NW] | (1u << I));
        }
        px.any |= nf;
    }
    px.any |= fin;
}

// Window rows [k_lo, T2_XIMG_R) of the tile whose first output row is oy.
template <int DT>
__device__ __forceinline__ void t2_load_x_t(const MhfdKHeader &h, const TcStretch &ts,
                                            unsigned char *x, const int *cmap, int oy, int k_lo, int wt) {
    constexpr int NCG = (T2_XIMG_C + 7) / 8;
    const int ITEMS = (T2_XIMG_R - k_lo) * NCG;
    constexpr int U = 2;
    const char *img = reinterpret_cast<const char *>(h.img);
#pragma unroll 1
    for (int i0 = wt; i0 < ITEMS; i0 += U * T2_NW) {
        // a group of 8 window columns maps to 8 consecutive image columns,
        // ascending, or (reflected at an edge) descending; only a group that
        // straddles an edge takes each column's index from the map
        unsigned raw[U][8];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = i0 + u * T2_NW;
            if (it < ITEMS) {
                const int kk = it / NCG, cg = it - kk * NCG, k = k_lo + kk;
                const char *row = img + (long long)reflect_idx(oy - 1 - RMAX + k, h.H) * h.pitch;
                const int g0 = cmap[8 * cg], g7 = cmap[8 * cg + 7];
                const int step = g0 >= 0 && g7 == g0 + 7 ? 1 : (MHFD_BOUNDARY == 0 && g7 >= 0 && g7 == g0 - 7 ? -1 : 0);
                if (step != 0) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) raw[u][e] = raw_px<DT>(row, g0 + step * e);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int gx = cmap[8 * cg + e];
                        raw[u][e] = gx >= 0 ? raw_px<DT>(row, gx) : (unsigned)ts.c0;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = i0 + u * T2_NW;
            if (it < ITEMS) {
                const int kk = it / NCG, cg = it - kk * NCG, k = k_lo + kk;
                unsigned pk[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2)
                    pk[e >> 1] = (unsigned)tc_px(raw[u][e], ts) | ((unsigned)tc_px(raw[u][e + 1], ts) << 16);
                if (mk_ok(cg < T2_XC / 8 && k < T2_XR))
                    *reinterpret_cast<uint4 *>(x + cg * T2_XGSTR + k * 16) =
                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
    }
}
// The tile's window: the column map first (image column of every window
// column, -1 past the window's image columns), then the rows.  When the
// tile is the one below the previous tile of the same strip (`below`), the
// previous window's rows from T2M - 2 on are this one's first rows: they move
// up in shared memory and only the rest is read from the image.
__device__ __forceinline__ void t2_load_x(const MhfdKHeader &h, const TcStretch &ts, const T2State &t,
                                          int oy, int ox, bool below, int wt) {
    constexpr int KEEP = T2_XIMG_R - (T2M - 2);  // rows shared with the tile above
    int *cmap = t.cmap();
    if (!below)
        for (int j = wt; j < T2_XC; j += T2_NW)
            cmap[j] = j < T2_XIMG_C ? reflect_idx(ox - 1 - RMAX + j, h.W) : -1;
    int k_lo = 0;
    if (below && KEEP > 0) {
        // rows [T2M - 2, T2_XIMG_R) to [0, KEEP): disjoint ranges, 16 bytes a row
        constexpr int NCG = (T2_XIMG_C + 7) / 8;
        unsigned char *x = t.xp();
        for (int i = wt; i < KEEP * NCG; i += T2_NW) {
            const int k = i % KEEP, cg = i / KEEP;
            if (mk_ok(cg < T2_XC / 8 && k + T2M - 2 < T2_XR))
                *reinterpret_cast<uint4 *>(x + cg * T2_XGSTR + k * 16) =
                    *reinterpret_cast<const uint4 *>(x + cg * T2_XGSTR + (k + T2M - 2) * 16);
        }
        k_lo = KEEP;
    }
    t2_wsync();
    if (h.dtype == 0)
        t2_load_x_t<0>(h, ts, t.xp(), cmap, oy, k_lo, wt);
    else
        t2_load_x_t<1>(h, ts, t.xp(), cmap, oy, k_lo, wt);
}

// The tile's candidate positions: each worker thread's count n goes to its
// row segment's rank in row-major order (cnt), a block scan forms their
// exclusive prefix (pre); returns the thread's first position, and the
// tile's total goes to tile_count[slot].
__device__ __forceinline__ int t2_count_scan(const MhfdKHeader &h, const T2State &t, int *cnt, int *pre, int n,
                                             int rank, long long slot, int wt) {
    const int w = wt >> 5, lane = wt & 31;
    if (mk_ok(rank >= 0 && rank < T2M * T2_CP)) cnt[rank] = n;
    t2_wsync();
    {
        constexpr int NWW = T2_NW / 32;
        static_assert(T2M * T2_CP == T2_NW, "one count per worker thread");
        const int v = cnt[wt];
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        int *buf = t.scan();
        if (lane == 31) buf[w] = x;
        t2_wsync();
        int before = 0, total = 0;
#pragma unroll
        for (int ww = 0; ww < NWW; ++ww) {
            const int tt = buf[ww];
            before += ww < w ? tt : 0;
            total += tt;
        }
        pre[wt] = before + x - v;
        if (wt == 0) h.tile_count[slot] = total;
    }
    t2_wsync();
    return pre[rank];
}

// The tile's maxima (Eq. 3 with the 3x3 test of §3) from the running max
// each worker thread holds for its row segment (TMEM lane m' = computed row
// 127 - m', columns CQ q .. CQ q + CQ - 1 reversed): the rows above and below
// are the neighbouring lanes (warp shuffles), the segment edges and the rows
// at the lane-group boundaries pass through shared memory (the split rows'
// space, free once the last horizontal product is done).  Candidates go to
// the tile's slots in row-major order (a scan of the per-segment counts in
// that order); the true count to tile_count.
__device__ __forceinline__ void t2_nms_regs(const MhfdKHeader &h, const T2State &t, const T2Tile &tl,
                                            T2Px &px, long long slot, int wt) {
    constexpr int CQ = T2_CQ;
    const float ninf = -__int_as_float(0x7f800000);
    float *xc = reinterpret_cast<float *>(t.ahp());  // [128 lanes][CP][2] segment edges
    float *xr = xc + T2M * T2_CP * 2;                 // [4 groups][2 ends][CP][CQ] boundary rows
    int *cnt = reinterpret_cast<int *>(xr + 8 * T2_CP * CQ);  // [128 rows][CP] counts, row-major
    int *pre = cnt + T2M * T2_CP;                              // their exclusive prefix
    const int w = wt >> 5, lane = wt & 31, g = w & 3, q = w >> 2;
    const int mr = 32 * g + lane;        // tensor-memory lane
    const int m = T2M - 1 - mr;          // computed row
    const int gy = tl.oy - 1 + m;
    const bool rowin = gy >= 0 && gy < h.H;
    // out-of-image pixels compare as -inf
#pragma unroll
    for (int u = 0; u < CQ; ++u) {
        const int gx = tl.ox - 1 + (TX2 - 1 - (CQ * q + u));
        if (!(rowin && gx >= 0 && gx < h.W)) px.mx[u] = ninf;
    }
    if (mk_ok(mr < T2M && q < T2_CP)) {
        xc[(mr * T2_CP + q) * 2 + 0] = px.mx[0];
        xc[(mr * T2_CP + q) * 2 + 1] = px.mx[CQ - 1];
    }
    if (lane == 0 || lane == 31) {
        float *dst = xr + ((g * 2 + (lane == 31 ? 1 : 0)) * T2_CP + q) * CQ;
#pragma unroll
        for (int u = 0; u < CQ; ++u) dst[u] = px.mx[u];
    }
    t2_wsync();
    // neighbour rows of lanes 0 and 31 (other lane groups; -inf past the tile)
    const float *rup = lane == 0 && g > 0 ? xr + (((g - 1) * 2 + 1) * T2_CP + q) * CQ : nullptr;
    const float *rdn = lane == 31 && g < 3 ? xr + (((g + 1) * 2 + 0) * T2_CP + q) * CQ : nullptr;
    // column max of the three rows just outside the segment (other part)
    auto edge = [&](int qq, int e) {
        if (qq < 0 || qq >= T2_CP) return ninf;
        float v = xc[(mr * T2_CP + qq) * 2 + e];
        if (mr > 0) v = fmaxf(v, xc[((mr - 1) * T2_CP + qq) * 2 + e]);
        if (mr < T2M - 1) v = fmaxf(v, xc[((mr + 1) * T2_CP + qq) * 2 + e]);
        return v;
    };
    float cprev = edge(q - 1, 1);  // n' = CQ q - 1
    const float cend = edge(q + 1, 0);  // n' = CQ q + CQ
    const float thr = h.thr;
    const bool rowint = rowin && m >= 1 && m <= T2M - 2;
    unsigned flags = 0;
    float vcur = 0.0f, ccur = 0.0f;  // column u: max of the rows above and below; of all three
#pragma unroll
    for (int u = 0; u <= CQ; ++u) {
        float vn = 0.0f, cn = cend;
        if (u < CQ) {
            // (volatile: the shuffles stay in column order, so the compiler
            // does not hold all of them in registers at once)
            float up, dn;
            asm volatile("shfl.sync.up.b32 %0, %1, 1, 0, 0xffffffff;" : "=f"(up) : "f"(px.mx[u]));
            asm volatile("shfl.sync.down.b32 %0, %1, 1, 31, 0xffffffff;" : "=f"(dn) : "f"(px.mx[u]));
            if (lane == 0) up = rup ? rup[u] : ninf;
            if (lane == 31) dn = rdn ? rdn[u] : ninf;
            vn = fmaxf(up, dn);
            cn = fmaxf(vn, px.mx[u]);
        }
        if (u > 0) {
            // pixel u - 1: its neighbours are the column maxima at u - 2 and u
            // and the rows above and below at u - 1
            const int uu = u - 1;
            const float x = px.mx[uu];
            const float nb = fmaxf(fmaxf(cprev, cn), vcur);
            const int c = TX2 - 1 - (CQ * q + uu);
            if (rowint && c >= 1 && c <= TX2 - 2 && x > thr && !(nb > x)) flags |= 1u << uu;
            cprev = ccur;
        }
        vcur = vn;
        ccur = cn;
    }
    // the flagged responses and argmaxes to shared memory (column u of
    // thread wt at [u][wt]), so that the writes below take a rolled loop
    float *smx = reinterpret_cast<float *>(t.ahp() + T2_NMS_VALS);
    unsigned char *sag = t.ahp() + T2_NMS_VALS + 4 * CQ * T2_NW;
#pragma unroll
    for (int u = 0; u < CQ; ++u)
        if (flags & (1u << u)) {
            smx[u * T2_NW + wt] = px.mx[u];
            sag[u * T2_NW + wt] = (unsigned char)t2_ag(px, u);
        }
    // positions: segments in row-major order (row m ascending, column
    // ascending = part descending)
    int pos = t2_count_scan(h, t, cnt, pre, __popc(flags), m * T2_CP + (T2_CP - 1 - q), slot, wt);
    if (flags && mk_ok(slot >= 0)) {
        MhfdCand *dst = h.stage + slot * h.cap_tile;
        // set bits from the highest column index u (lowest image column)
#pragma unroll 1
        for (unsigned f = flags; f; ++pos) {
            const int uu = 31 - __clz(f);
            f &= ~(1u << uu);
            if (pos < h.cap_tile) {
                MhfdCand cd;
                cd.x = tl.ox - 1 + (TX2 - 1 - (CQ * q + uu));
                cd.y = gy;
                cd.i = sag[uu * T2_NW + wt];
                cd.resp = smx[uu * T2_NW + wt];
                dst[pos] = cd;
            }
        }
    }
    if (STORE && rowint) {
#pragma unroll
        for (int uu = 0; uu < CQ; ++uu) {
            const int c = TX2 - 1 - (CQ * q + uu);
            const int gx = tl.ox - 1 + c;
            if (c >= 1 && c <= TX2 - 2 && gx < h.W && mk_ok(gx >= 0)) {
                const long long o2 = (long long)gy * h.W + gx;
                if (h.m_out) h.m_out[o2] = px.mx[uu];
                if (h.arg_out) h.arg_out[o2] = t2_ag(px, uu);
            }
        }
    }
    t2_wsync();  // the exchange space is the next tile's split rows
}

// The tile's kept items of the 26-neighbour rule to its slots: row-major
// order, layers ascending within a pixel (the order of the other kernels),
// by a scan of the per-segment counts; responses from the block's scratch.
// The masks are cleared for the next tile.  The counts use the split rows'
// space, free once the last horizontal product is done.
__device__ __forceinline__ void t2_out26(const MhfdKHeader &h, const T2State &t, const T2Tile &tl, T2Px &px,
                                         long long slot, int wt) {
    constexpr int CQ = T2_CQ;
    const int w = wt >> 5, lane = wt & 31, g = w & 3, q = w >> 2;
    const int m = T2M - 1 - (32 * g + lane);
    int *cnt = reinterpret_cast<int *>(t.ahp());  // [128 rows][CP] counts, row-major
    int *pre = cnt + T2M * T2_CP;                 // their exclusive prefix
    unsigned short *msk = t.l26m() + wt;
    constexpr long long LAY = (long long)CQ * T2_NW;
    const float *gv = h.l26val + (long long)blockIdx.x * (NL - 1) * LAY + wt;
    int n = 0;
#pragma unroll 1
    for (unsigned f = px.any; f; f &= f - 1) n += __popc(msk[(__ffs(f) - 1) * T2_NW]);
    int pos = t2_count_scan(h, t, cnt, pre, n, m * T2_CP + (T2_CP - 1 - q), slot, wt);
    MhfdCand *dst = h.stage + slot * h.cap_tile;
    // columns from the highest u (lowest image column)
#pragma unroll 1
    for (unsigned f = px.any; f;) {
        const int uu = 31 - __clz(f);
        f &= ~(1u << uu);
        unsigned mm = msk[uu * T2_NW];
        msk[uu * T2_NW] = 0;
#pragma unroll 1
        for (; mm; mm &= mm - 1, ++pos)
            if (pos < h.cap_tile && mk_ok(slot >= 0)) {
                const int i = __ffs(mm) - 1;
                MhfdCand cd;
                cd.x = tl.ox - 1 + (TX2 - 1 - (CQ * q + uu));
                cd.y = tl.oy - 1 + m;
                cd.i = i;
                cd.resp = gv[i * LAY + uu * T2_NW];
                dst[pos] = cd;
            }
    }
    px.any = 0;
    t2_wsync();  // the count space is the next tile's split rows
}

// worker levels: wait for level l's V, split it, build level l + 2's tap
// matrix, hand over; then the responses of level l - 1
// (after the last level's split, the last vertical product is done: the
// next tile's window loads then, so the tensor core runs this tile's last
// horizontal product and the next tile's first vertical ones while the
// workers finish this tile's responses and maxima)
__device__ __forceinline__ void t2_work(const MhfdKHeader &h, T2State &t, const TcStretch &ts, T2Px &px,
                                        const T2Tile &tl, bool next, const T2Tile &tn, int wt) {
#pragma unroll 1
    for (int l = 0; l < NL; ++l) {
        const unsigned gl = t.g + (unsigned)l;
        t2_wait(h, t, T2_VB + (int)(gl & 1u));
        if (l > 0) t2_wait(h, t, T2_HB + (int)((gl - 1u) & 1u));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        t2_split(t, l, (gl & 1u) * (unsigned)T2_NVMAX, wt);
        t2_arrive(t2_bar(t, T2_SPL));
        if (l == NL - 1 && next) {
            t2_load_x(h, ts, t, tn.oy, tn.ox, tn.ox == tl.ox && tn.oy == tl.oy + TY, wt);
            t2_arrive(t2_bar(t, T2_XRB));
        }
        if (l > 0) {
            const unsigned dcol = (unsigned)T2_DH + ((gl - 1u) & 1u) * (unsigned)TX2;
            if constexpr (T2_L26)
                t2_epi26(h, t, l - 1, dcol, px, ts.a, tl);
            else
                t2_epi(h, t, l - 1, dcol, wt, px, ts.a, tl);
        }
    }
}

// issuer levels: after level l's split, level l's horizontal product and
// level l + 2's vertical one
// (level l's tap matrices are fetched three levels ahead, into the buffer
// that level l - 1 used: its horizontal product is done once the workers
// have split level l; the last three levels fetch the next tile's first)
__device__ __forceinline__ void t2_issue(const MhfdKHeader &h, T2State &t, bool next) {
#pragma unroll 1
    for (int l = 0; l < NL; ++l) {
        const unsigned gl = t.g + (unsigned)l;
        t2_wait(h, t, T2_SPL);
        __syncwarp();  // converged for elect.sync
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (l + 3 < NL)
            t2_fetch_tab(h, t, l + 3, gl + 3u);
        else if (next)
            t2_fetch_tab(h, t, l + 3 - NL, gl + 3u);
        t2_issue_h(t, l, t2_tabb(t, gl), (unsigned)T2_DH + (gl & 1u) * (unsigned)TX2);
        t2_commit(t2_bar(t, T2_HB + (int)(gl & 1u)));
        if (l + 2 < NL) {
            t2_wait(h, t, T2_TB + (int)((gl + 2u) % (unsigned)T2_NTAB));
            __syncwarp();
            t2_issue_v(t, l + 2, t2_tabb(t, gl + 2u), (gl & 1u) * (unsigned)T2_NVMAX);
            t2_commit(t2_bar(t, T2_VB + (int)(gl & 1u)));
        }
    }
}

__device__ __forceinline__ T2Tile t2_tile(long long k, int tiles_y) {
    T2Tile tl;
    const int tx = (int)(k / tiles_y), ty = (int)(k - (long long)tx * tiles_y);
    tl.oy = ty * TY;
    tl.ox = tx * TX;
    return tl;
}

// Tiles [k0, k1) of an image (strip-major order), tile k's candidates into
// slot slot0 + (its tile row) * tiles_x + (its strip).
__device__ __forceinline__ void t2_range(const MhfdKHeader &h, long long k0, long long k1, int tiles_x,
                                         int tiles_y, long long slot0, T2State &t) {
    if (k0 >= k1) return;
    const MhfdStretch st = *h.st;
    TcStretch ts = tc_stretch(st);
    ts.a = st.inv * (1.0f / (T2_S * T2_S));
    if (threadIdx.x >= T2_NW) {
#pragma unroll 1
        // the first tile's first three tap matrices (the buffers are free:
        // the previous range's products are done)
        for (int l = 0; l < 3; ++l) t2_fetch_tab(h, t, l, t.g + (unsigned)l);
        for (long long k = k0; k < k1; ++k) {
            t2_wait(h, t, T2_XRB);
            __syncwarp();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            t2_wait(h, t, T2_TB + (int)(t.g % (unsigned)T2_NTAB));
            __syncwarp();
            t2_issue_v(t, 0, t2_tabb(t, t.g), ((t.g & 1u) * (unsigned)T2_NVMAX));
            t2_commit(t2_bar(t, T2_VB + (int)(t.g & 1u)));
            t2_wait(h, t, T2_TB + (int)((t.g + 1u) % (unsigned)T2_NTAB));
            __syncwarp();
            t2_issue_v(t, 1, t2_tabb(t, t.g + 1u), (((t.g + 1u) & 1u) * (unsigned)T2_NVMAX));
            t2_commit(t2_bar(t, T2_VB + (int)((t.g + 1u) & 1u)));
            t2_issue(h, t, k + 1 < k1);
            t.g += NL;
        }
        return;
    }
    const int wt = threadIdx.x;
    {
        const T2Tile t0 = t2_tile(k0, tiles_y);
        t2_load_x(h, ts, t, t0.oy, t0.ox, false, wt);
        t2_arrive(t2_bar(t, T2_XRB));
    }
#pragma unroll 1
    for (long long k = k0; k < k1; ++k) {
        const T2Tile tl = t2_tile(k, tiles_y);
        const bool next = k + 1 < k1;
        const T2Tile tn = t2_tile(next ? k + 1 : k, tiles_y);
        T2Px px;
        t2_work(h, t, ts, px, tl, next, tn, wt);
        const unsigned gl = t.g + NL - 1;
        t2_wait(h, t, T2_HB + (int)(gl & 1u));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned dcol = (unsigned)T2_DH + (gl & 1u) * (unsigned)TX2;
        const int tx = (int)(k / tiles_y), ty = (int)(k - (long long)tx * tiles_y);
        const long long slot = slot0 + (long long)ty * tiles_x + tx;
        if constexpr (T2_L26) {
            // the top layer's items, then the tile's kept items to its slots
            t2_epi26(h, t, NL - 1, dcol, px, ts.a, tl);
            t2_out26(h, t, tl, px, slot, wt);
        } else {
            // the tile's maxima (Eq. 3 with the 3x3 test of §3) from the
            // responses in registers
            t2_epi(h, t, NL - 1, dcol, wt, px, ts.a, tl);
            t2_nms_regs(h, t, tl, px, slot, wt);
        }
        t.g += NL;
    }
}
#endif  // MHFD_VTC == 2

// Tiles [k0, k1) of an image in strip-major order (k -> strip k / tiles_y,
// tile row k % tiles_y), as one march per strip touched.
__device__ __forceinline__ void run_range(const MhfdKHeader &h, long long k0, long long k1,
                                          int tiles_x, int tiles_y, long long slot0,
                                          const Smem &sm, TcState &tc) {
    const MhfdStretch st = *h.st;
    long long k = k0;
    while (k < k1) {
        const int tx = (int)(k / tiles_y);
        const int ta = (int)(k - (long long)tx * tiles_y);
        const int tb = (int)min((long long)tiles_y, ta + (k1 - k));
        if constexpr (TC)
            march_tc(h, st, tiles_x, tx, ta, tb, slot0, sm, tc);
        else
            march(h, st, tiles_x, tx, ta, tb, slot0, sm);
        k += tb - ta;
    }
}

// batch: persistent blocks take chunks of `chunk` tiles from the queue
// (no waits); chunk -> (job, tiles) through chunk_base
__device__ __forceinline__ void batch_loop(const KParams &p, const Smem &sm, TcState &tc) {
    __shared__ int s_item;
#pragma unroll 1
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(p.h.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= p.h.total_items) break;
        int lo = 0, hi = p.h.n_jobs - 1;  // last job with chunk_base <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.h.jobs[mid].chunk_base <= item) lo = mid; else hi = mid - 1;
        }
        const MhfdJob job = p.h.jobs[lo];
        // gated batches: the tensor-core launch takes the images whose
        // stretch range it holds exactly, the FFMA launch the others
        if (p.h.gate != 0 && (p.h.gate == 1) != tc_narrow(job.dtype, *job.st)) continue;
        MhfdKHeader h = p.h;
        h.img = job.img;
        h.st = job.st;
        h.pitch = job.pitch;
        h.H = job.H;
        h.W = job.W;
        h.dtype = job.dtype;
        h.tiles_x = job.tiles_x;
        h.tiles_y = job.tiles_y;
        h.plane = (long long)job.H * job.W;
        const long long n_tiles = (long long)job.tiles_x * job.tiles_y;
        const long long k0 = (long long)(item - job.chunk_base) * p.h.chunk;
        const long long k1 = min(n_tiles, k0 + p.h.chunk);
        run_range(h, k0, k1, job.tiles_x, job.tiles_y, job.tile_base, sm, tc);
    }
}

}  // namespace mk

#if MHFD_VTC == 2
namespace mk {
// The two-pass kernel's block: shared-memory layout, mbarriers and tensor
// memory, then a single image's share of tiles or the batch queue.
__device__ __forceinline__ void t2_kernel(const KParams &p, unsigned char *base) {
    __shared__ int s_item;
    if (p.h.dtype == 2) {  // float images never reach this kernel
        if (threadIdx.x == 0 && p.h.flag) atomicOr(p.h.flag, 1);
        return;
    }
    T2State t;
    unsigned char *ctrl = t.ctrl();  // 10 mbarriers, TMEM address (+96), fail flag (+100)
    // the window's padding rows and columns stay zero; the 26-neighbour
    // rule's layer masks start empty (each tile's end clears what it read)
    for (int i = threadIdx.x; i < T2_X_BYTES / 16; i += NT)
        reinterpret_cast<uint4 *>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (T2_L26)
        for (int i = threadIdx.x; i < 2 * TX2 * T2M / 16; i += NT)
            reinterpret_cast<uint4 *>(t.l26m())[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 10; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(ctrl + 8 * b)),
                         "r"(b == T2_SPL || b == T2_XRB ? T2_NW / 32 : 1)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *reinterpret_cast<volatile int *>(ctrl + 100) = 0;
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(ctrl + 96)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    t.tmem = *reinterpret_cast<volatile unsigned *>(ctrl + 96);
    t.ph = 0;
    t.g = 0;
    if (p.h.jobs == nullptr) {
        const bool run = p.h.gate == 0 || ((p.h.gate == 1) == tc_narrow(p.h.dtype, *p.h.st));
        const long long T = (long long)p.h.tiles_x * p.h.tiles_y;
        const long long k0 = T * blockIdx.x / gridDim.x;
        const long long k1 = T * (blockIdx.x + 1) / gridDim.x;
        if (run) t2_range(p.h, k0, k1, p.h.tiles_x, p.h.tiles_y, 0, t);
    } else {
#pragma unroll 1
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) s_item = atomicAdd(p.h.queue, 1);
            __syncthreads();
            const int item = s_item;
            if (item >= p.h.total_items) break;
            int lo = 0, hi = p.h.n_jobs - 1;  // last job with chunk_base <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.h.jobs[mid].chunk_base <= item) lo = mid; else hi = mid - 1;
            }
            const MhfdJob job = p.h.jobs[lo];
            if (p.h.gate != 0 && (p.h.gate == 1) != tc_narrow(job.dtype, *job.st)) continue;
            MhfdKHeader h = p.h;
            h.img = job.img;
            h.st = job.st;
            h.pitch = job.pitch;
            h.H = job.H;
            h.W = job.W;
            h.dtype = job.dtype;
            h.tiles_x = job.tiles_x;
            h.tiles_y = job.tiles_y;
            h.plane = (long long)job.H * job.W;
            const long long n_tiles = (long long)job.tiles_x * job.tiles_y;
            const long long k0 = (long long)(item - job.chunk_base) * p.h.chunk;
            const long long k1 = min(n_tiles, k0 + p.h.chunk);
            if (job.dtype == 2) continue;
            t2_range(h, k0, k1, job.tiles_x, job.tiles_y, job.tile_base, t);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(512u)
                     : "memory");
}
}  // namespace mk
#endif

#if MHFD_VTC == 2
// The two-pass kernel's banded tap matrices of every level, in the layout of
// its shared-memory buffers (hi part, then lo part at T2_TAB_PART): block l
// writes level l.  Run once per detector; the kernel copies one level at a
// time.
extern "C" __constant__ int mhfd_t2_tab_bytes = mk::NL * 2 * mk::T2_TAB_PART;
extern "C" __global__ void __launch_bounds__(mk::T2_NW) mhfd_t2_tables(unsigned char *out) {
    using namespace mk;
    const int l = blockIdx.x;
    if (l >= NL || blockDim.x != T2_NW) return;
    unsigned char *tab = out + (long long)l * (2 * T2_TAB_PART);
    for (int i = threadIdx.x; i < 2 * T2_TAB_PART / 16; i += T2_NW)
        reinterpret_cast<uint4 *>(tab)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    t2_build_tab(tab, l, threadIdx.x);
}
#endif

extern "C" __global__ void __launch_bounds__(mk::NT, 1)
    mhfd_fused_detect(const __grid_constant__ mk::KParams p) {
    using namespace mk;
    extern __shared__ __align__(16) float smem[];
#if MHFD_VTC == 2
    t2_kernel(p, reinterpret_cast<unsigned char *>(smem));
    return;
#endif
    Smem sm;
    if constexpr (TC) {
        sm.win = reinterpret_cast<unsigned char *>(smem);
        sm.btab = sm.win + TC_WIN_BYTES;
        sm.in = nullptr;
        sm.v = reinterpret_cast<float *>(sm.btab + TC_B_BYTES);
    } else {
        sm.win = sm.btab = nullptr;
        sm.in = smem;
        sm.v = smem + SMEM_IN;
    }
    sm.ring = sm.v + SMEM_V;
    sm.arg = reinterpret_cast<unsigned char *>(sm.ring + SMEM_RING_F);
    sm.scan = reinterpret_cast<int *>(sm.arg + SMEM_RING_B);
    sm.ctrl = reinterpret_cast<unsigned char *>(sm.scan) + 4 * 64;

    if constexpr (CHECKS) {
        if (threadIdx.x == 0) mk_chk_flag = p.h.flag;
        __syncthreads();
    }
    // single image with a gate: the tensor-core kernel takes narrow stretch
    // ranges, its FFMA companion the rest (both launched, one works); a batch
    // applies the gate per image
    if (p.h.jobs == nullptr && p.h.gate != 0) {
        const bool narrow = tc_narrow(p.h.dtype, *p.h.st);
        if ((p.h.gate == 1) != narrow) return;
    }
    TcState tc{};
    if constexpr (TC) {
        if (p.h.dtype == 2) {  // float images never reach this kernel
            if (threadIdx.x == 0 && p.h.flag) atomicOr(p.h.flag, 1);
            return;
        }
        tc_setup_smem(sm.win, sm.btab);
        unsigned *tslot = reinterpret_cast<unsigned *>(sm.ctrl + 96);
        if (threadIdx.x == 0) {
            for (int g = 0; g < NGROUPS; ++g)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(sm.ctrl + 8 * g))
                             : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_addr(tslot)),
                         "r"((unsigned)TC_TCOLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tc.tmem = *tslot;
        tc.win = smem_addr(sm.win);
        tc.btab = smem_addr(sm.btab);
        tc.bar = smem_addr(sm.ctrl);
        tc.ph = 0;
        tc.issuer = threadIdx.x == TC_ISSUER;
    }

    if (p.h.jobs == nullptr) {
        // one image: block b takes an equal share of its tiles
        const long long T = (long long)p.h.tiles_x * p.h.tiles_y;
        const long long k0 = T * blockIdx.x / gridDim.x;
        const long long k1 = T * (blockIdx.x + 1) / gridDim.x;
        run_range(p.h, k0, k1, p.h.tiles_x, p.h.tiles_y, 0, sm, tc);
    } else {
        batch_loop(p, sm, tc);
    }
    if constexpr (TC) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (threadIdx.x < 32)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem),
                         "r"((unsigned)TC_TCOLS)
                         : "memory");
    }
}

