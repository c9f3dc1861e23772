// Device helpers shared by the overlap-prune kernels (post.cu, noalloc.cu).
#ifndef MHFD_PRUNE_COMMON_CUH
#define MHFD_PRUNE_COMMON_CUH

#include "mhfd_types.h"

namespace mhfd {
namespace {

// Fraction of the smaller circle covered by the lens of two circles, in the
// same operation order as the CPU oracle (round-to-nearest, no contraction).
__device__ __forceinline__ double lens_overlap(double r1, double r2, double d) {
    const double rmin = r1 < r2 ? r1 : r2;
    if (d >= __dadd_rn(r1, r2)) return 0.0;
    if (d <= fabs(__dsub_rn(r1, r2))) return 1.0;
    const double dd = __dmul_rn(d, d), r11 = __dmul_rn(r1, r1), r22 = __dmul_rn(r2, r2);
    double a1 = __ddiv_rn(__dsub_rn(__dadd_rn(dd, r11), r22), __dmul_rn(__dmul_rn(2.0, d), r1));
    double a2 = __ddiv_rn(__dsub_rn(__dadd_rn(dd, r22), r11), __dmul_rn(__dmul_rn(2.0, d), r2));
    a1 = a1 > 1.0 ? 1.0 : (a1 < -1.0 ? -1.0 : a1);
    a2 = a2 > 1.0 ? 1.0 : (a2 < -1.0 ? -1.0 : a2);
    const double f1 = __dadd_rn(__dadd_rn(-d, r1), r2);
    const double f2 = __dsub_rn(__dadd_rn(d, r1), r2);
    const double f3 = __dadd_rn(__dsub_rn(d, r1), r2);
    const double f4 = __dadd_rn(__dadd_rn(d, r1), r2);
    double k = __dmul_rn(__dmul_rn(__dmul_rn(f1, f2), f3), f4);
    if (k < 0.0) k = 0.0;
    const double area = __dsub_rn(__dadd_rn(__dmul_rn(r11, acos(a1)), __dmul_rn(r22, acos(a2))),
                                  __dmul_rn(0.5, __dsqrt_rn(k)));
    return __ddiv_rn(area, __dmul_rn(__dmul_rn(3.14159265358979323846, rmin), rmin));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool higher(const MhfdCand &b, const MhfdCand &a, int W) {
    if (b.i != a.i) return b.i > a.i;
    if (b.resp != a.resp) return b.resp > a.resp;
    return (long long)b.y * W + b.x < (long long)a.y * W + a.x;
}

}  // namespace
}  // namespace mhfd

#endif  // MHFD_PRUNE_COMMON_CUH
