// Complex FP64 helpers (double2 = re, im) and the per-panel 2x2 block-Jacobi
// preconditioner shared by the GMRES drivers.
#pragma once

#include <cuda_runtime.h>

namespace lspr {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Right preconditioner of panel i: the inverse of the diagonal 2x2 block of the operator,
// [[1/2 + K_ii, -V_ii], [1/2 - K_ii, s V_ii]] with K_ii = 0:
//   [[1/2, -V], [1/2, s V]]^-1 = [[s V, V], [-1/2, 1/2]] / (V (1 + s) / 2)
__device__ __forceinline__ void block_jacobi(double V, double2 s, double2 u0, double2 u1, double2 &o0, double2 &o1) {
    const double2 det = make_double2(0.5 * V * (1.0 + s.x), 0.5 * V * s.y);
    const double2 a = cadd(cmul(cscale(s, V), u0), cscale(u1, V));
    const double2 c = make_double2(0.5 * (u1.x - u0.x), 0.5 * (u1.y - u0.y));
    o0 = cdiv(a, det);
    o1 = cdiv(c, det);
}

}  // namespace lspr
