/*
 * FP64 CPU oracle of Multi-scale Histologic Feature Detection (MHFD).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path: every step below is written
 * straight from the paper's definitions, in plain loops, in double precision,
 * in the order the paper states them.  Speed is not a goal.
 *
 * Steps and the passages they follow:
 *   stretch   - §3, histogram stretching: saturate 0.175 % of the darkest and
 *               0.175 % of the lightest pixels and map the range to [0, 1]
 *               (Algorithm 1, first step).
 *   ladder    - §2.2: n, min_t, max_t, dt = (max_t - min_t)/n,
 *               t_i = min_t + (i-1) dt, here for i = 1 .. n+1.
 *   kernel    - §2.2: isotropic Gaussian of variance t^2, sampled on the pixel
 *               grid, truncated at R = ceil(truncate * t), normalised to sum 1.
 *   blur      - §2.2: L(., t) = G(., t) * I', done as a separable direct
 *               convolution (columns, then rows), reflect boundary
 *               ("d c b a | a b c d | d c b a") or periodic boundary.
 *   dog       - Eq. 2: DoG(x, y, i) = t_i (L(x, y, t_{i+1}) - L(x, y, t_i)).
 *   nms       - Eq. 3 and §3: inner argmax over all scales (first index on
 *               ties), outer spatial local maximum by comparison with a 3x3
 *               max-pool (non-strict, out-of-image neighbours ignored), kept
 *               when the response exceeds the threshold.  A 26-neighbour
 *               (3x3x3) scale-space local-maximum mode is also provided.
 *   prune     - greedy overlap pruning (not in the paper): blobs of radius
 *               sqrt(2) t_i, visited by radius desc, response desc, linear
 *               index asc; a blob is dropped when an already kept blob covers
 *               more than `overlap` of the smaller circle's area.
 *   score     - §3 / Algorithm 1: the criterion is the number of features.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by the per-pixel loops (each output pixel is computed by one
 * thread in a fixed order, so the result does not depend on this). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define OR_U8 0
#define OR_U16 1
#define OR_F32 2

#define OR_REFLECT 0
#define OR_PERIODIC 1

static double value_at(const void *img, int dtype, int64_t row_stride_bytes, int64_t y, int64_t x) {
    const unsigned char *row = (const unsigned char *)img + y * row_stride_bytes;
    if (dtype == OR_U8) return (double)row[x];
    if (dtype == OR_U16) return (double)((const uint16_t *)row)[x];
    return (double)((const float *)row)[x];
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* §3 histogram stretch: k = floor(clip * N); lo is the k-th smallest value
 * (0-based order statistic) and hi the (N-1-k)-th smallest. */
int oracle_stretch_bounds(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                          double clip, double *lo, double *hi) {
    int64_t N = H * W;
    if (N <= 0) return -1;
    double *v = (double *)malloc((size_t)N * sizeof(double));
    if (!v) return -2;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) v[y * W + x] = value_at(img, dtype, row_stride_bytes, y, x);
    qsort(v, (size_t)N, sizeof(double), cmp_double);
    int64_t k = (int64_t)floor(clip * (double)N);   /* 0 <= clip < 0.5 */
    *lo = v[k];
    *hi = v[N - 1 - k];
    free(v);
    return 0;
}

/* §3: I' = min(max((I - lo) / (hi - lo), 0), 1); a constant image (hi == lo)
 * maps to 0. */
void oracle_stretch(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                    double lo, double hi, double *out) {
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            double v = value_at(img, dtype, row_stride_bytes, y, x);
            double s = 0.0;
            if (hi > lo) {
                s = (v - lo) / (hi - lo);
                if (s < 0.0) s = 0.0;
                if (s > 1.0) s = 1.0;
            }
            out[y * W + x] = s;
        }
}

/* §2.2 scale ladder, i = 1 .. n+1 stored at t[0 .. n]. */
void oracle_ladder(int n, double tmin, double tmax, double *t) {
    double dt = (tmax - tmin) / (double)n;
    for (int i = 1; i <= n + 1; ++i) t[i - 1] = tmin + (double)(i - 1) * dt;
}

int oracle_kernel_radius(double t, double truncate) { return (int)ceil(truncate * t); }

/* §2.2 sampled Gaussian of std t on k = -R .. R (stored at g[k + R]),
 * normalised so that the taps sum to one. */
void oracle_kernel(double t, int R, double *g) {
    double sum = 0.0;
    for (int k = -R; k <= R; ++k) {
        g[k + R] = exp(-((double)k * (double)k) / (2.0 * t * t));
        sum += g[k + R];
    }
    for (int k = -R; k <= R; ++k) g[k + R] /= sum;
}

static int64_t boundary_index(int64_t i, int64_t N, int boundary) {
    if (boundary == OR_PERIODIC) {
        int64_t m = i % N;
        return m < 0 ? m + N : m;
    }
    /* reflect about the pixel edges: period 2N, second half mirrored */
    int64_t p = 2 * N;
    int64_t m = i % p;
    if (m < 0) m += p;
    return m < N ? m : p - 1 - m;
}

/* §2.2 blur: out = g (x) g applied to `in`; first along columns (y), then
 * along rows (x). */
void oracle_blur(const double *in, int64_t H, int64_t W, const double *g, int R, int boundary,
                 double *out) {
    double *tmp = (double *)malloc((size_t)(H * W) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int k = -R; k <= R; ++k) acc += g[k + R] * in[boundary_index(y + k, H, boundary) * W + x];
            tmp[y * W + x] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int k = -R; k <= R; ++k) acc += g[k + R] * tmp[y * W + boundary_index(x + k, W, boundary)];
            out[y * W + x] = acc;
        }
    free(tmp);
}

/* Eq. 2 over the ladder t[0..n]: D[i] = t_i (L_{i+1} - L_i) for i = 0..n-1
 * (0-based), D laid out as n planes of H x W. */
void oracle_dog_stack(const double *Ip, int64_t H, int64_t W, const double *t, int n,
                      double truncate, int boundary, double *D) {
    int64_t P = H * W;
    double *Lprev = (double *)malloc((size_t)P * sizeof(double));
    double *Lcur = (double *)malloc((size_t)P * sizeof(double));
    for (int i = 0; i <= n; ++i) {
        int R = oracle_kernel_radius(t[i], truncate);
        double *g = (double *)malloc((size_t)(2 * R + 1) * sizeof(double));
        oracle_kernel(t[i], R, g);
        oracle_blur(Ip, H, W, g, R, boundary, Lcur);
        free(g);
        if (i > 0)
            for (int64_t p = 0; p < P; ++p) D[(int64_t)(i - 1) * P + p] = t[i - 1] * (Lcur[p] - Lprev[p]);
        double *sw = Lprev; Lprev = Lcur; Lcur = sw;
    }
    free(Lprev);
    free(Lcur);
}

/* §2.2, the response the DoG approximates: the scale-normalised Laplacian
 * t_i^2 grad^2 L(., t_i), i = 0..n-1 (scales t_1..t_n), with the Laplacian
 * discretised by the 5-point stencil on the level (neighbours through the
 * same boundary as the blur).  D laid out as n planes of H x W. */
void oracle_log_stack(const double *Ip, int64_t H, int64_t W, const double *t, int n,
                      double truncate, int boundary, double *D) {
    int64_t P = H * W;
    double *L = (double *)malloc((size_t)P * sizeof(double));
    for (int i = 0; i < n; ++i) {
        int R = oracle_kernel_radius(t[i], truncate);
        double *g = (double *)malloc((size_t)(2 * R + 1) * sizeof(double));
        oracle_kernel(t[i], R, g);
        oracle_blur(Ip, H, W, g, R, boundary, L);
        free(g);
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                const double c = L[y * W + x];
                const double lap = L[y * W + boundary_index(x - 1, W, boundary)] +
                                   L[y * W + boundary_index(x + 1, W, boundary)] +
                                   L[boundary_index(y - 1, H, boundary) * W + x] +
                                   L[boundary_index(y + 1, H, boundary) * W + x] - 4.0 * c;
                D[(int64_t)i * P + y * W + x] = t[i] * t[i] * lap;
            }
    }
    free(L);
}

/* Eq. 3, the paper's mode: M = max_i D_i, i_hat = first maximiser; (x, y)
 * is kept when M > thr and M >= M at every in-image 8-neighbour (comparison
 * with a 3x3 max-pool).  Returns the number of features; writes at most
 * `cap` of them. */
int64_t oracle_nms_paper(const double *D, int n, int64_t H, int64_t W, double thr,
                         int32_t *ox, int32_t *oy, int32_t *oi, double *oresp, int64_t cap) {
    int64_t P = H * W;
    double *M = (double *)malloc((size_t)P * sizeof(double));
    int32_t *A = (int32_t *)malloc((size_t)P * sizeof(int32_t));
    for (int64_t p = 0; p < P; ++p) {
        double best = D[p];
        int arg = 0;
        for (int i = 1; i < n; ++i)
            if (D[(int64_t)i * P + p] > best) { best = D[(int64_t)i * P + p]; arg = i; }
        M[p] = best;
        A[p] = arg;
    }
    int64_t count = 0;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            double m = M[y * W + x];
            if (!(m > thr)) continue;
            int ok = 1;
            for (int dy = -1; dy <= 1 && ok; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    if (M[yy * W + xx] > m) { ok = 0; break; }
                }
            if (!ok) continue;
            if (count < cap) {
                ox[count] = (int32_t)x; oy[count] = (int32_t)y; oi[count] = A[y * W + x];
                oresp[count] = m;
            }
            ++count;
        }
    free(M);
    free(A);
    return count;
}

/* 26-neighbour mode: (x, y, i) is kept when D_i(x, y) > thr and it is >= every
 * neighbour in the 3x3x3 scale-space window that lies inside the stack. */
int64_t oracle_nms_local26(const double *D, int n, int64_t H, int64_t W, double thr,
                           int32_t *ox, int32_t *oy, int32_t *oi, double *oresp, int64_t cap) {
    int64_t P = H * W;
    int64_t count = 0;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x)
            for (int i = 0; i < n; ++i) {
                double v = D[(int64_t)i * P + y * W + x];
                if (!(v > thr)) continue;
                int ok = 1;
                for (int di = -1; di <= 1 && ok; ++di)
                    for (int dy = -1; dy <= 1 && ok; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int64_t ii = i + di, yy = y + dy, xx = x + dx;
                            if (ii < 0 || ii >= n || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            if (D[ii * P + yy * W + xx] > v) { ok = 0; break; }
                        }
                if (!ok) continue;
                if (count < cap) {
                    ox[count] = (int32_t)x; oy[count] = (int32_t)y; oi[count] = i; oresp[count] = v;
                }
                ++count;
            }
    return count;
}

/* Fraction of the smaller circle covered by the intersection (lens) of two
 * circles of radii r1, r2 whose centres are d apart: 1 when one contains the
 * other, 0 when they are disjoint. */
double oracle_lens_overlap(double r1, double r2, double d) {
    double rmin = r1 < r2 ? r1 : r2;
    if (d >= r1 + r2) return 0.0;
    if (d <= fabs(r1 - r2)) return 1.0;
    double a1 = (d * d + r1 * r1 - r2 * r2) / (2.0 * d * r1);
    double a2 = (d * d + r2 * r2 - r1 * r1) / (2.0 * d * r2);
    if (a1 > 1.0) a1 = 1.0;
    if (a1 < -1.0) a1 = -1.0;
    if (a2 > 1.0) a2 = 1.0;
    if (a2 < -1.0) a2 = -1.0;
    double k = (-d + r1 + r2) * (d + r1 - r2) * (d - r1 + r2) * (d + r1 + r2);
    if (k < 0.0) k = 0.0;
    double area = r1 * r1 * acos(a1) + r2 * r2 * acos(a2) - 0.5 * sqrt(k);
    return area / (M_PI * rmin * rmin);
}

/* oracle_lens_overlap over m (r1, r2, d) triples (for checks over many pairs). */
void oracle_lens_overlap_many(const double *r1, const double *r2, const double *d, int64_t m,
                              double *out) {
    for (int64_t j = 0; j < m; ++j) out[j] = oracle_lens_overlap(r1[j], r2[j], d[j]);
}

/* priority order of the greedy prune */
typedef struct {
    int32_t x, y, i;
    double resp;
    int64_t lin;
    int64_t idx;
} or_item;

static int cmp_priority(const void *pa, const void *pb) {
    const or_item *a = (const or_item *)pa, *b = (const or_item *)pb;
    if (a->i != b->i) return a->i > b->i ? -1 : 1;             /* radius desc */
    if (a->resp != b->resp) return a->resp > b->resp ? -1 : 1; /* response desc */
    if (a->lin != b->lin) return a->lin < b->lin ? -1 : 1;     /* linear index asc */
    return 0;
}

/* Greedy overlap prune.  radius[i] is the blob radius of scale index i.
 * keep[j] = 1 for survivors.  A uniform bucket grid of kept blobs is used
 * only to skip pairs farther apart than r1 + r2 (whose overlap is zero). */
int64_t oracle_prune(const int32_t *x, const int32_t *y, const int32_t *si, const double *resp,
                     int64_t n, const double *radius, int n_levels, double overlap, int64_t W,
                     uint8_t *keep) {
    if (n <= 0) return 0;
    or_item *it = (or_item *)malloc((size_t)n * sizeof(or_item));
    double rmax = 0.0;
    for (int i = 0; i < n_levels; ++i) if (radius[i] > rmax) rmax = radius[i];
    int32_t xmax = 0, ymax = 0;
    for (int64_t j = 0; j < n; ++j) {
        it[j].x = x[j]; it[j].y = y[j]; it[j].i = si[j]; it[j].resp = resp[j];
        it[j].lin = (int64_t)y[j] * W + x[j]; it[j].idx = j;
        keep[j] = 0;
        if (x[j] > xmax) xmax = x[j];
        if (y[j] > ymax) ymax = y[j];
    }
    qsort(it, (size_t)n, sizeof(or_item), cmp_priority);
    double cell = 2.0 * rmax + 1.0;
    int64_t ncx = (int64_t)(xmax / cell) + 1, ncy = (int64_t)(ymax / cell) + 1;
    int64_t *head = (int64_t *)malloc((size_t)(ncx * ncy) * sizeof(int64_t));
    int64_t *next = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t c = 0; c < ncx * ncy; ++c) head[c] = -1;
    int64_t kept = 0;
    for (int64_t a = 0; a < n; ++a) {
        const or_item *p = &it[a];
        double rp = radius[p->i];
        int64_t cx = (int64_t)(p->x / cell), cy = (int64_t)(p->y / cell);
        int drop = 0;
        for (int64_t gy = cy - 1; gy <= cy + 1 && !drop; ++gy)
            for (int64_t gx = cx - 1; gx <= cx + 1 && !drop; ++gx) {
                if (gx < 0 || gy < 0 || gx >= ncx || gy >= ncy) continue;
                for (int64_t b = head[gy * ncx + gx]; b >= 0; b = next[b]) {
                    const or_item *q = &it[b];
                    double dx = (double)(p->x - q->x), dy = (double)(p->y - q->y);
                    double d = sqrt(dx * dx + dy * dy);
                    if (oracle_lens_overlap(radius[q->i], rp, d) > overlap) { drop = 1; break; }
                }
            }
        if (drop) continue;
        keep[p->idx] = 1;
        ++kept;
        int64_t c = cy * ncx + cx;
        next[a] = head[c];
        head[c] = a;
    }
    free(head);
    free(next);
    free(it);
    return kept;
}

/* Response stack at one pixel: D_i(x, y) for i = 0..n-1 straight from the raw
 * image (stretch, then for each scale the 2-D separable sum over the
 * (2R+1)^2 window with reflect boundary).  Used for spot checks at sizes
 * where the full stack would be slow. */
void oracle_dog_at(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                   double lo, double hi, const double *t, int n, double truncate, int64_t x,
                   int64_t y, double *Dout) {
    double Lprev = 0.0;
    for (int i = 0; i <= n; ++i) {
        int R = oracle_kernel_radius(t[i], truncate);
        double *g = (double *)malloc((size_t)(2 * R + 1) * sizeof(double));
        oracle_kernel(t[i], R, g);
        double acc = 0.0;
        for (int ky = -R; ky <= R; ++ky) {
            int64_t yy = boundary_index(y + ky, H, OR_REFLECT);
            for (int kx = -R; kx <= R; ++kx) {
                int64_t xx = boundary_index(x + kx, W, OR_REFLECT);
                double v = value_at(img, dtype, row_stride_bytes, yy, xx);
                double s = 0.0;
                if (hi > lo) {
                    s = (v - lo) / (hi - lo);
                    if (s < 0.0) s = 0.0;
                    if (s > 1.0) s = 1.0;
                }
                acc += g[ky + R] * g[kx + R] * s;
            }
        }
        free(g);
        if (i > 0) Dout[i - 1] = t[i - 1] * (acc - Lprev);
        Lprev = acc;
    }
}

/* Adjoint (transpose) of oracle_blur: out = B^T in for B = rows o columns.
 * Every value in[y][x] is scattered with weight g[k] to the input positions
 * the forward pass read it from; the transpose of the row pass comes first,
 * then the transpose of the column pass.  With the reflect boundary the
 * mirrored reads scatter back to their mirrored sources. */
void oracle_blur_adjoint(const double *in, int64_t H, int64_t W, const double *g, int R,
                         int boundary, double *out) {
    double *tmp = (double *)calloc((size_t)(H * W), sizeof(double));
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            const double v = in[y * W + x];
            for (int k = -R; k <= R; ++k) tmp[y * W + boundary_index(x + k, W, boundary)] += g[k + R] * v;
        }
    for (int64_t p = 0; p < H * W; ++p) out[p] = 0.0;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            const double v = tmp[y * W + x];
            for (int k = -R; k <= R; ++k) out[boundary_index(y + k, H, boundary) * W + x] += g[k + R] * v;
        }
    free(tmp);
}

/* Soft focus score over the ladder t[0..n] (n DoG layers), the stretch
 * bounds lo/hi held fixed:
 *   S = sum_i w_i mean_{x,y} sigmoid((D_i(x,y) - tau) / T),  D_i of Eq. 2.
 * mean_sig[i] receives mean_{x,y} sigmoid(...) (= dS/dw_i).  If dimg is not
 * NULL it receives dS/dI in input units by the exact transpose of every
 * linear step: dD_i = w_i s (1 - s) / (T N); dL_l = t_{l-1} dD_{l-1} -
 * t_l dD_l; dI' = sum_l B_l^T dL_l; dI = dI' / (hi - lo) where lo < I < hi
 * (the clamp of the stretch passes nothing elsewhere).  Returns S. */
double oracle_soft_score(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                         double lo, double hi, const double *t, int n, double truncate, double tau,
                         double T, const double *w, double *mean_sig, double *dimg) {
    const int64_t P = H * W;
    double *Ip = (double *)malloc((size_t)P * sizeof(double));
    oracle_stretch(img, dtype, H, W, row_stride_bytes, lo, hi, Ip);
    double *L = (double *)malloc((size_t)(P * (n + 1)) * sizeof(double));
    int *Rs = (int *)malloc((size_t)(n + 1) * sizeof(int));
    double **G = (double **)malloc((size_t)(n + 1) * sizeof(double *));
    for (int l = 0; l <= n; ++l) {
        Rs[l] = oracle_kernel_radius(t[l], truncate);
        G[l] = (double *)malloc((size_t)(2 * Rs[l] + 1) * sizeof(double));
        oracle_kernel(t[l], Rs[l], G[l]);
        oracle_blur(Ip, H, W, G[l], Rs[l], OR_REFLECT, L + (int64_t)l * P);
    }
    double S = 0.0;
    double *gD = dimg ? (double *)calloc((size_t)(P * n), sizeof(double)) : NULL;
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t p = 0; p < P; ++p) {
            const double d = t[i] * (L[(int64_t)(i + 1) * P + p] - L[(int64_t)i * P + p]);
            const double sg = 1.0 / (1.0 + exp(-(d - tau) / T));
            acc += sg;
            if (gD) gD[(int64_t)i * P + p] = w[i] * sg * (1.0 - sg) / (T * (double)P);
        }
        mean_sig[i] = acc / (double)P;
        S += w[i] * mean_sig[i];
    }
    if (dimg) {
        double *h = (double *)malloc((size_t)P * sizeof(double));
        double *adj = (double *)malloc((size_t)P * sizeof(double));
        double *gI = (double *)calloc((size_t)P, sizeof(double));
        for (int l = 0; l <= n; ++l) {
            for (int64_t p = 0; p < P; ++p) {
                double v = 0.0;
                if (l >= 1) v += t[l - 1] * gD[(int64_t)(l - 1) * P + p];
                if (l <= n - 1) v -= t[l] * gD[(int64_t)l * P + p];
                h[p] = v;
            }
            oracle_blur_adjoint(h, H, W, G[l], Rs[l], OR_REFLECT, adj);
            for (int64_t p = 0; p < P; ++p) gI[p] += adj[p];
        }
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                const double v = value_at(img, dtype, row_stride_bytes, y, x);
                dimg[y * W + x] = (hi > lo && v > lo && v < hi) ? gI[y * W + x] / (hi - lo) : 0.0;
            }
        free(h);
        free(adj);
        free(gI);
        free(gD);
    }
    for (int l = 0; l <= n; ++l) free(G[l]);
    free(G);
    free(Rs);
    free(L);
    free(Ip);
    return S;
}

/* oracle_dog_at for a list of pixels; D laid out [m][n]. */
void oracle_dog_at_many(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                        double lo, double hi, const double *t, int n, double truncate,
                        const int64_t *xs, const int64_t *ys, int64_t m, double *D) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < m; ++j)
        oracle_dog_at(img, dtype, H, W, row_stride_bytes, lo, hi, t, n, truncate, xs[j], ys[j],
                      D + j * n);
}

int64_t oracle_detect_ex(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                         int n, double tmin, double tmax, double truncate, double clip, double thr,
                         double overlap, int mode, int response, int boundary, int32_t *cx,
                         int32_t *cy, int32_t *ci, double *cresp, uint8_t *keep, int64_t cap,
                         int64_t *n_kept, double *lo_out, double *hi_out);

/* Whole method on one image (Algorithm 1 without distribution, plus the
 * threshold and the prune): stretch, ladder, stack, NMS, prune.
 * mode 0 = the paper's argmax/max-pool, 1 = 26-neighbour.
 * Candidates are written to (cx, cy, ci, cresp) up to `cap`; keep[] flags the
 * survivors.  Returns the true candidate count; *n_kept receives the number
 * of survivors (among the written candidates); lo/hi are returned too. */
int64_t oracle_detect(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                      int n, double tmin, double tmax, double truncate, double clip, double thr,
                      double overlap, int mode, int32_t *cx, int32_t *cy, int32_t *ci, double *cresp,
                      uint8_t *keep, int64_t cap, int64_t *n_kept, double *lo_out, double *hi_out) {
    return oracle_detect_ex(img, dtype, H, W, row_stride_bytes, n, tmin, tmax, truncate, clip, thr,
                            overlap, mode, 0, OR_REFLECT, cx, cy, ci, cresp, keep, cap, n_kept,
                            lo_out, hi_out);
}

/* As oracle_detect with a choice of response (0: DoG of Eq. 2, 1: the
 * scale-normalised Laplacian t^2 grad^2 L) and boundary (reflect/periodic). */
int64_t oracle_detect_ex(const void *img, int dtype, int64_t H, int64_t W, int64_t row_stride_bytes,
                         int n, double tmin, double tmax, double truncate, double clip, double thr,
                         double overlap, int mode, int response, int boundary, int32_t *cx,
                         int32_t *cy, int32_t *ci, double *cresp, uint8_t *keep, int64_t cap,
                         int64_t *n_kept, double *lo_out, double *hi_out) {
    double lo, hi;
    if (oracle_stretch_bounds(img, dtype, H, W, row_stride_bytes, clip, &lo, &hi) != 0) return -1;
    *lo_out = lo;
    *hi_out = hi;
    double *Ip = (double *)malloc((size_t)(H * W) * sizeof(double));
    oracle_stretch(img, dtype, H, W, row_stride_bytes, lo, hi, Ip);
    double *t = (double *)malloc((size_t)(n + 1) * sizeof(double));
    oracle_ladder(n, tmin, tmax, t);
    double *D = (double *)malloc((size_t)(H * W) * (size_t)n * sizeof(double));
    if (response == 1)
        oracle_log_stack(Ip, H, W, t, n, truncate, boundary, D);
    else
        oracle_dog_stack(Ip, H, W, t, n, truncate, boundary, D);
    int64_t cnt = mode == 0 ? oracle_nms_paper(D, n, H, W, thr, cx, cy, ci, cresp, cap)
                            : oracle_nms_local26(D, n, H, W, thr, cx, cy, ci, cresp, cap);
    double *radius = (double *)malloc((size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) radius[i] = sqrt(2.0) * t[i];
    int64_t m = cnt < cap ? cnt : cap;
    *n_kept = oracle_prune(cx, cy, ci, cresp, m, radius, n, overlap, W, keep);
    free(radius);
    free(D);
    free(t);
    free(Ip);
    return cnt;
}
