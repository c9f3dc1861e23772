// Fused multi-scale feature detection kernel (sm_103a).
//
// Compiled at run time with NVRTC once per ladder: the host prepends MHFD_*
// macros (number of Gaussian levels, their radii, the f32 tap values and
// scale factors as exact hexadecimal literals, tile geometry, mode) so that
// every loop over scales and taps is fully unrolled and every tap is an
// immediate operand of its FFMA (no constant-memory load per multiply).
//
// One CTA produces the features of one (TY x TX) output tile:
//   1. load the tile plus a halo of RMAX+1 pixels from global memory (reflect
//      boundary: "d c b a | a b c d | d c b a"), apply the histogram stretch
//      of §3 on the fly and keep the f32 block in shared memory;
//   2. march over the tile in steps of RB rows.  Per step and per group of
//      levels, a vertical pass computes V_l = g_l (*)_y I' for every column of
//      the halo'd width: each thread owns a column, forms the folded sums
//      I'(y+k) + I'(y-k) once and feeds them to all levels of the group
//      (taps are symmetric, §2.2), for up to four rows at a time;
//   3. a horizontal pass computes L_l = g_l (*)_x V_l for four adjacent
//      outputs per thread from float4 shared-memory reads and forms the DoG
//      of Eq. 2, D_{l-1} = t_{l-1} (L_l - L_{l-1}), in registers;
//   4. the paper's rule (Eq. 3) keeps the running max over scales and its
//      first argmax in registers and compares it with its 3x3 neighbourhood
//      from a (RB+2)-row ring in shared memory; the 26-neighbour mode keeps a
//      ring of the whole response stack instead;
//   5. features above the threshold are compacted in tile order (block scan)
//      into the tile's slots of the candidate list.
// The response stack never reaches global memory (except in the STORE
// variant used by the tests).

#ifndef MHFD_NL
#error "MHFD_* configuration macros must be defined before this source"
#endif

namespace mk {

#define MK_HD __host__ __device__

constexpr int NL = MHFD_NL;
constexpr int NDOG = NL - 1;
constexpr int NGROUPS = MHFD_NGROUPS;
constexpr int TX2 = MHFD_TX2;
constexpr int TX = TX2 - 2;
constexpr int TY2 = MHFD_TY2;
constexpr int TY = TY2 - 2;
constexpr int RB = MHFD_RB;
constexpr int NT = MHFD_NT;
constexpr int MODE = MHFD_MODE;  // 0: paper (argmax over scales + 3x3), 1: 3x3x3
constexpr bool STORE = (MHFD_STORE) != 0;

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
template <int I>
__device__ __forceinline__ float tap() {
    constexpr float v = kTap(I);
    return v;
}
MK_HD constexpr int rmax_of() {
    int m = 0;
    for (int l = 0; l < NL; ++l) m = kR(l) > m ? kR(l) : m;
    return m;
}
constexpr int RMAX = rmax_of();
constexpr int WEXT = TX2 + 2 * RMAX;           // columns of the halo'd block
constexpr int WEXTP = (WEXT + 3) & ~3;
constexpr int ROWS_IN = TY2 + 2 * RMAX;        // rows of the halo'd block
constexpr int NSTEPS = TY2 / RB;
constexpr int RING = RB + 2;
constexpr int NQ4 = TX2 / 4;
constexpr int HITEMS = RB * NQ4;
constexpr int HI = (HITEMS + NT - 1) / NT;
constexpr int NPARTS = (RB + 3) / 4;

// padded width of the V row of level l (its outputs plus its own halo)
MK_HD constexpr int extp(int l) { return (TX2 + 2 * kR(l) + 3) & ~3; }
// taps of level l start at tapoff(l) of the parameter block
MK_HD constexpr int tapoff(int l) {
    int o = 0;
    for (int j = 0; j < l; ++j) o += kR(j) + 1;
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
    for (int j = kGB(group_of(l)); j < l; ++j) o += extp(j);
    return o;
}
MK_HD constexpr int vrow_max() {
    int m = 0;
    for (int g = 0; g < NGROUPS; ++g) {
        int o = 0;
        for (int j = kGB(g); j < kGB(g + 1); ++j) o += extp(j);
        m = o > m ? o : m;
    }
    return m;
}
constexpr int NTAPS = tapoff(NL);
constexpr int VROW = vrow_max();
constexpr int SMEM_IN = ROWS_IN * WEXTP;
constexpr int SMEM_V = RB * VROW;
constexpr int SMEM_RING_F = MODE == 0 ? RING * TX2 : RING * NDOG * TX2;
constexpr int SMEM_RING_B = MODE == 0 ? ((RING * TX2 + 15) & ~15) : 0;
constexpr int SMEM_BYTES = 4 * (SMEM_IN + SMEM_V + SMEM_RING_F) + SMEM_RING_B + 4 * 64;

static_assert(TX2 % 4 == 0, "tile width must be a multiple of 4");
static_assert(TY2 % RB == 0, "tile height must be a multiple of the step");
static_assert(NT % 32 == 0 && NT <= 1024, "threads per block");
static_assert(NL >= 2 && NL <= 64, "levels");
static_assert(kGB(0) == 0 && kGB(NGROUPS) == NL, "level groups");

struct KParams {
    MhfdKHeader h;
};

struct HState {
    float lp[4];  // L of the previous level
    float m[4];   // running max over scales
    int a[4];     // its first argmax
};

__device__ __forceinline__ int reflect_idx(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

// ---------------------------------------------------------------- 1. load

template <int DT>
__device__ __forceinline__ float load_px(const char *row, int gx, const MhfdStretch &st) {
    if (DT == 0) {
        int v = __ldg(reinterpret_cast<const unsigned char *>(row) + gx);
        v = min(max(v, st.lo_i), st.hi_i);
        return fmaf((float)(v - st.lo_i), st.inv, st.off);
    } else if (DT == 1) {
        int v = __ldg(reinterpret_cast<const unsigned short *>(row) + gx);
        v = min(max(v, st.lo_i), st.hi_i);
        return fmaf((float)(v - st.lo_i), st.inv, st.off);
    } else {
        const float v = __ldg(reinterpret_cast<const float *>(row) + gx);
        float u = (v - st.lo) * st.inv;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        return u + st.off;
    }
}

template <int DT>
__device__ __forceinline__ void load_block(const MhfdKHeader &h, const MhfdStretch &st, float *s_in,
                                           int x0, int y0) {
    // each thread owns columns; LB row loads are kept in flight at a time so
    // that the latency of the global (mostly L2) reads overlaps
    constexpr int LB = 16;
    const char *base = reinterpret_cast<const char *>(h.img);
    const long long pitch = h.pitch;
    const int H = h.H, W = h.W;
    for (int c = threadIdx.x; c < WEXT; c += NT) {
        const int gx = reflect_idx(x0 - 1 - RMAX + c, W);
        float *dst = s_in + c;
        int r = 0;
#pragma unroll 1
        for (; r + LB <= ROWS_IN; r += LB) {
            float v[LB];
#pragma unroll
            for (int e = 0; e < LB; ++e) {
                const int gy = reflect_idx(y0 - 1 - RMAX + r + e, H);
                v[e] = load_px<DT>(base + (long long)gy * pitch, gx, st);
            }
#pragma unroll
            for (int e = 0; e < LB; ++e) dst[(r + e) * WEXTP] = v[e];
        }
        for (; r < ROWS_IN; ++r) {
            const int gy = reflect_idx(y0 - 1 - RMAX + r, H);
            dst[r * WEXTP] = load_px<DT>(base + (long long)gy * pitch, gx, st);
        }
    }
}

// Fold step K of the vertical pass for the levels L.. of group G: every
// level whose radius reaches K takes tap K times the folded sum.
template <int G, int K, int L>
__device__ __forceinline__ void vlev(float sum, float *a) {
    constexpr int LB = kGB(G);
    constexpr int NG = kGB(G + 1) - LB;
    if constexpr (L < NG) {
        if constexpr (K <= kR(LB + L)) a[L] = fmaf(tap<tapoff(LB + L) + K>(), sum, a[L]);
        vlev<G, K, L + 1>(sum, a);
    }
}

template <int G, int L>
__device__ __forceinline__ void vinit(float x, float *a) {
    constexpr int LB = kGB(G);
    constexpr int NG = kGB(G + 1) - LB;
    if constexpr (L < NG) {
        a[L] = tap<tapoff(LB + L)>() * x;
        vinit<G, L + 1>(x, a);
    }
}

template <int G, int ROWS, int K>
__device__ __forceinline__ void vstep(const float *colp, float (*acc)[kGB(G + 1) - kGB(G)]) {
    if constexpr (K <= kR(kGB(G + 1) - 1)) {
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const float sum = colp[(j + K) * WEXTP] + colp[(j - K) * WEXTP];
            vlev<G, K, 0>(sum, acc[j]);
        }
        vstep<G, ROWS, K + 1>(colp, acc);
    }
}

// V_l(o0 + j, c) for the ROWS rows starting at tile row o0 and every level l
// of group G.  Row o of the tile sits at row o + RMAX of the halo'd block.
template <int G, int ROWS>
__device__ __forceinline__ void vcol(const MhfdKHeader &h, const float *__restrict__ s_in,
                                     float *__restrict__ s_v, int c, int o0, int jb) {
    constexpr int LB = kGB(G);
    constexpr int LE = kGB(G + 1);
    constexpr int NG = LE - LB;
    float acc[ROWS][NG];
    const float *colp = s_in + (o0 + RMAX) * WEXTP + c;
#pragma unroll
    for (int j = 0; j < ROWS; ++j) vinit<G, 0>(colp[j * WEXTP], acc[j]);
    vstep<G, ROWS, 1>(colp, acc);
#pragma unroll
    for (int l = 0; l < NG; ++l) {
        const int cc = c - (RMAX - kR(LB + l));
        if (cc >= 0 && cc < TX2 + 2 * kR(LB + l)) {
#pragma unroll
            for (int j = 0; j < ROWS; ++j) s_v[(jb + j) * VROW + voff(LB + l) + cc] = acc[j][l];
        }
    }
}

template <int G, int PART>
struct VParts {
    static __device__ __forceinline__ void run(const MhfdKHeader &h, const float *s_in, float *s_v,
                                               int c, int s) {
        constexpr int ROWS = (RB - 4 * PART) < 4 ? (RB - 4 * PART) : 4;
        vcol<G, ROWS>(h, s_in, s_v, c, s * RB + 4 * PART, 4 * PART);
        VParts<G, PART + 1>::run(h, s_in, s_v, c, s);
    }
};
template <int G>
struct VParts<G, NPARTS> {
    static __device__ __forceinline__ void run(const MhfdKHeader &, const float *, float *, int, int) {}
};

template <int G>
__device__ __forceinline__ void vpass(const MhfdKHeader &h, const float *s_in, float *s_v, int s) {
#pragma unroll 1
    for (int c = threadIdx.x; c < WEXT; c += NT) VParts<G, 0>::run(h, s_in, s_v, c, s);
}

// ----------------------------------------------------- 3. horizontal pass

// value number M of the window feeds output U with tap |M - U - R|
template <int R, int TO, int M, int U>
__device__ __forceinline__ void hacc1(float v, float (&a)[4]) {
    constexpr int k = M - U - R;
    if constexpr (k >= -R && k <= R) a[U] = fmaf(tap<TO + (k < 0 ? -k : k)>(), v, a[U]);
}

template <int R, int TO, int M>
__device__ __forceinline__ void hacc(const MhfdKHeader &, float v, float (&a)[4]) {
    hacc1<R, TO, M, 0>(v, a);
    hacc1<R, TO, M, 1>(v, a);
    hacc1<R, TO, M, 2>(v, a);
    hacc1<R, TO, M, 3>(v, a);
}

template <int R, int TO, int M4>
struct HQuads {
    static __device__ __forceinline__ void run(const MhfdKHeader &h, const float4 *w, float (&a)[4]) {
        const float4 v = w[M4];
        hacc<R, TO, 4 * M4 + 0>(h, v.x, a);
        hacc<R, TO, 4 * M4 + 1>(h, v.y, a);
        hacc<R, TO, 4 * M4 + 2>(h, v.z, a);
        hacc<R, TO, 4 * M4 + 3>(h, v.w, a);
        HQuads<R, TO, M4 - 1>::run(h, w, a);
    }
};
template <int R, int TO>
struct HQuads<R, TO, -1> {
    static __device__ __forceinline__ void run(const MhfdKHeader &, const float4 *, float (&)[4]) {}
};

struct HCtx {
    int r;        // tile row of this item
    int q;        // float4 chunk (outputs 4q .. 4q+3)
    int slot;     // ring slot of row r
    int gy;       // image row
    int gx0;      // image column of output 4q
    bool inb[4];  // output inside the image
    bool inter[4];  // output inside the tile interior and the image (stored)
};

template <int L>
__device__ __forceinline__ void hlevel(const MhfdKHeader &h, const float *vrow, const HCtx &cx,
                                       HState &st, float *s_ring) {
    constexpr int R = kR(L);
    constexpr int NQ = (2 * R + 3) / 4 + 1;
    float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const float4 *w = reinterpret_cast<const float4 *>(vrow + voff(L)) + cx.q;
    HQuads<R, tapoff(L), NQ - 1>::run(h, w, a);
    if (L == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            st.lp[u] = a[u];
            st.m[u] = -__int_as_float(0x7f800000);
            st.a[u] = 0;
        }
    } else {
        constexpr int I = (L > 0 ? L - 1 : 0);
        constexpr float ts = kTsc(I);
        float d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            d[u] = ts * (a[u] - st.lp[u]);
            st.lp[u] = a[u];
        }
        if (MODE == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (d[u] > st.m[u]) {
                    st.m[u] = d[u];
                    st.a[u] = I;
                }
        } else {
            const float ninf = -__int_as_float(0x7f800000);
            float4 o;
            o.x = cx.inb[0] ? d[0] : ninf;
            o.y = cx.inb[1] ? d[1] : ninf;
            o.z = cx.inb[2] ? d[2] : ninf;
            o.w = cx.inb[3] ? d[3] : ninf;
            reinterpret_cast<float4 *>(s_ring + (cx.slot * NDOG + I) * TX2)[cx.q] = o;
        }
        if (STORE) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cx.inter[u])
                    h.stack_out[(long long)I * h.plane + (long long)cx.gy * h.W + cx.gx0 + u] =
                        d[u];
        }
    }
}

template <int L, int LE>
struct HLevels {
    static __device__ __forceinline__ void run(const MhfdKHeader &h, const float *vrow,
                                               const HCtx &cx, HState &st, float *s_ring) {
        hlevel<L>(h, vrow, cx, st, s_ring);
        HLevels<L + 1, LE>::run(h, vrow, cx, st, s_ring);
    }
};
template <int LE>
struct HLevels<LE, LE> {
    static __device__ __forceinline__ void run(const MhfdKHeader &, const float *, const HCtx &,
                                               HState &, float *) {}
};

__device__ __forceinline__ HCtx make_ctx(const MhfdKHeader &h, int item, int s, int x0, int y0) {
    HCtx cx;
    const int j = item / NQ4;
    cx.q = item - j * NQ4;
    cx.r = s * RB + j;
    cx.slot = cx.r % RING;
    cx.gy = y0 - 1 + cx.r;
    cx.gx0 = x0 - 1 + 4 * cx.q;
    const bool rowin = cx.gy >= 0 && cx.gy < h.H;
    const bool rowint = rowin && cx.r >= 1 && cx.r <= TY2 - 2;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int gx = cx.gx0 + u;
        const int c = 4 * cx.q + u;
        cx.inb[u] = rowin && gx >= 0 && gx < h.W;
        cx.inter[u] = rowint && c >= 1 && c <= TX2 - 2 && gx < h.W;
    }
    return cx;
}

template <int G>
__device__ __forceinline__ void hpass(const MhfdKHeader &h, const float *s_v, float *s_ring,
                                      unsigned char *s_arg, HState (&hs)[HI], int s, int x0,
                                      int y0) {
#pragma unroll
    for (int it = 0; it < HI; ++it) {
        const int item = threadIdx.x + it * NT;
        if (item < HITEMS) {
            const HCtx cx = make_ctx(h, item, s, x0, y0);
            const float *vrow = s_v + (cx.r - s * RB) * VROW;
            HLevels<kGB(G), kGB(G + 1)>::run(h, vrow, cx, hs[it], s_ring);
            if (G == NGROUPS - 1 && MODE == 0) {
                const float ninf = -__int_as_float(0x7f800000);
                float4 o;
                o.x = cx.inb[0] ? hs[it].m[0] : ninf;
                o.y = cx.inb[1] ? hs[it].m[1] : ninf;
                o.z = cx.inb[2] ? hs[it].m[2] : ninf;
                o.w = cx.inb[3] ? hs[it].m[3] : ninf;
                reinterpret_cast<float4 *>(s_ring + cx.slot * TX2)[cx.q] = o;
                uchar4 ab;
                ab.x = (unsigned char)hs[it].a[0];
                ab.y = (unsigned char)hs[it].a[1];
                ab.z = (unsigned char)hs[it].a[2];
                ab.w = (unsigned char)hs[it].a[3];
                reinterpret_cast<uchar4 *>(s_arg + cx.slot * TX2)[cx.q] = ab;
                if (STORE) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (cx.inter[u]) {
                            const long long o2 = (long long)cx.gy * h.W + cx.gx0 + u;
                            if (h.m_out) h.m_out[o2] = hs[it].m[u];
                            if (h.arg_out) h.arg_out[o2] = hs[it].a[u];
                        }
                }
            }
        }
    }
}

template <int G>
struct Groups {
    static __device__ __forceinline__ void run(const MhfdKHeader &h, const float *s_in, float *s_v,
                                               float *s_ring, unsigned char *s_arg,
                                               HState (&hs)[HI], int s, int x0, int y0) {
        vpass<G>(h, s_in, s_v, s);
        __syncthreads();
        hpass<G>(h, s_v, s_ring, s_arg, hs, s, x0, y0);
        __syncthreads();
        Groups<G + 1>::run(h, s_in, s_v, s_ring, s_arg, hs, s, x0, y0);
    }
};
template <>
struct Groups<NGROUPS> {
    static __device__ __forceinline__ void run(const MhfdKHeader &, const float *, float *, float *,
                                               unsigned char *, HState (&)[HI], int, int, int) {}
};

// ------------------------------------------------------ 4-5. NMS, compaction

// exclusive block scan of one int per thread; *sum receives the total
__device__ __forceinline__ int block_excl_scan(int v, int *s_scan, int *sum) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NW ? s_scan[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_scan[lane] = w;
    }
    __syncthreads();
    const int excl = (warp > 0 ? s_scan[warp - 1] : 0) + x - v;
    *sum = s_scan[NW - 1];
    __syncthreads();
    return excl;
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

// 26-neighbour rule on the response ring
__device__ __forceinline__ bool cand_26(const float *s_ring, int r, int c, int l, float thr,
                                        float *v_out) {
    const float v = s_ring[((r % RING) * NDOG + l) * TX2 + c];
    *v_out = v;
    if (!(v > thr)) return false;
#pragma unroll
    for (int dl = -1; dl <= 1; ++dl) {
        const int ll = l + dl;
        if (ll < 0 || ll >= NDOG) continue;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
            const float *row = s_ring + (((r + dr) % RING) * NDOG + ll) * TX2;
            if (row[c - 1] > v || row[c] > v || row[c + 1] > v) return false;
        }
    }
    return true;
}

__device__ __forceinline__ int nms_step(const MhfdKHeader &h, const float *s_ring,
                                        const unsigned char *s_arg, int *s_scan, int s, int x0,
                                        int y0, int tile, int total) {
    const int r_lo = max(1, s * RB - 1);
    const int r_hi = min(TY2 - 2, s * RB + RB - 2);
    if (r_lo > r_hi) return total;
    const int nrows = r_hi - r_lo + 1;
    const int per = (MODE == 0) ? TX : TX * NDOG;
    const int items = nrows * per;
    const int ch = (items + NT - 1) / NT;
    const int beg = min(items, (int)threadIdx.x * ch);
    const int end = min(items, beg + ch);
    const float thr = h.thr;
    int cnt = 0;
    for (int it = beg; it < end; ++it) {
        const int r = r_lo + it / per;
        const int rem = it - (it / per) * per;
        float v;
        if (MODE == 0) {
            cnt += cand_paper(s_ring, r, 1 + rem, thr, &v) ? 1 : 0;
        } else {
            cnt += cand_26(s_ring, r, 1 + rem / NDOG, rem % NDOG, thr, &v) ? 1 : 0;
        }
    }
    int sum;
    int pos = total + block_excl_scan(cnt, s_scan, &sum);
    if (cnt) {
        MhfdCand *dst = h.stage + (long long)tile * h.cap_tile;
        for (int it = beg; it < end; ++it) {
            const int r = r_lo + it / per;
            const int rem = it - (it / per) * per;
            float v;
            bool ok;
            int c, l;
            if (MODE == 0) {
                c = 1 + rem;
                ok = cand_paper(s_ring, r, c, thr, &v);
                l = s_arg[(r % RING) * TX2 + c];
            } else {
                c = 1 + rem / NDOG;
                l = rem % NDOG;
                ok = cand_26(s_ring, r, c, l, thr, &v);
            }
            if (ok) {
                if (pos < h.cap_tile) {
                    MhfdCand cd;
                    cd.x = x0 - 1 + c;
                    cd.y = y0 - 1 + r;
                    cd.i = l;
                    cd.resp = v;
                    dst[pos] = cd;
                }
                ++pos;
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

// The whole detection of one output tile (load, stack, DoG, maxima,
// compaction).  `item` indexes the candidate slots and counts.
__device__ __forceinline__ void process_tile(const MhfdKHeader &h, int tile,
                                             int item, float *s_in, float *s_v, float *s_ring,
                                             unsigned char *s_arg, int *s_scan) {
    const int ty = tile / h.tiles_x;
    const int tx = tile - ty * h.tiles_x;
    const int x0 = tx * TX, y0 = ty * TY;
    const MhfdStretch st = *h.st;

    if (h.dtype == 0)
        load_block<0>(h, st, s_in, x0, y0);
    else if (h.dtype == 1)
        load_block<1>(h, st, s_in, x0, y0);
    else
        load_block<2>(h, st, s_in, x0, y0);
    __syncthreads();

    HState hs[HI];
    int total = 0;
#pragma unroll 1
    for (int s = 0; s < NSTEPS; ++s) {
        Groups<0>::run(h, s_in, s_v, s_ring, s_arg, hs, s, x0, y0);
        total = nms_step(h, s_ring, s_arg, s_scan, s, x0, y0, item, total);
    }
    if (threadIdx.x == 0) h.tile_count[item] = total;
}

}  // namespace mk

extern "C" __global__ void __launch_bounds__(mk::NT, 1)
    mhfd_fused_detect(const __grid_constant__ mk::KParams p) {
    using namespace mk;
    extern __shared__ __align__(16) float smem[];
    float *s_in = smem;
    float *s_v = smem + SMEM_IN;
    float *s_ring = s_v + SMEM_V;
    unsigned char *s_arg = reinterpret_cast<unsigned char *>(s_ring + SMEM_RING_F);
    int *s_scan = reinterpret_cast<int *>(s_arg + SMEM_RING_B);

    if (p.h.jobs == nullptr) {
        process_tile(p.h, blockIdx.x, blockIdx.x, s_in, s_v, s_ring, s_arg, s_scan);
        return;
    }
    // batch: persistent blocks take items from the queue (no waits)
    __shared__ int s_item;
#pragma unroll 1
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(p.h.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= p.h.total_items) break;
        int lo = 0, hi = p.h.n_jobs - 1;  // last job with tile_base <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.h.jobs[mid].tile_base <= item) lo = mid; else hi = mid - 1;
        }
        const MhfdJob job = p.h.jobs[lo];
        MhfdKHeader h = p.h;
        h.img = job.img;
        h.st = job.st;
        h.pitch = job.pitch;
        h.H = job.H;
        h.W = job.W;
        h.dtype = job.dtype;
        h.tiles_x = job.tiles_x;
        h.plane = (long long)job.H * job.W;
        process_tile(h, item - job.tile_base, item, s_in, s_v, s_ring, s_arg, s_scan);
    }
}
