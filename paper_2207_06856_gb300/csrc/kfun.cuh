// Kernel functions evaluated from a pre-scaled negative squared distance.
//
// Both MVM engines feed the kernel function s = -c^2 r^2 / 2, where the
// inputs were scaled by c / l_k before the distance was formed:
//   RBF        c = sqrt(log2 e)  ->  s = -log2(e) r^2 / 2,  k = 2^s
//   Matern-3/2 c = sqrt(6)       ->  s = -3 r^2,  u = sqrt(-s) = sqrt3 r,  k = (1 + u) e^-u
//   Matern-1/2 c = sqrt(2)       ->  s = -r^2,    u = r,                    k = e^-u
//   Matern-5/2 c = sqrt(10)      ->  s = -5 r^2,  u = sqrt5 r,              k = (1 + u + u^2/3) e^-u
// so RBF costs one ex2 and the Matern kernels one sqrt and one ex2 on the
// special function units.  s can come out slightly positive for coincident
// points (rounding); RBF then returns 2^s ~ 1, the Matern forms clamp u at 0.
#pragma once
#include "ptx.cuh"
#include "../../include/gpk.h"

namespace gpk {

constexpr float kLog2e = 1.4426950408889634f;

template <int KIND>
__device__ __forceinline__ float kernel_from_s(float s) {
    if constexpr (KIND == GP_KERNEL_RBF) {
        return ptx::ex2(s);
    } else {
        const float u = ptx::sqrt_approx(fmaxf(-s, 0.0f));
        const float e = ptx::ex2(-kLog2e * u);
        if constexpr (KIND == GP_KERNEL_MATERN32) {
            return fmaf(u, e, e);
        } else if constexpr (KIND == GP_KERNEL_MATERN12) {
            return e;
        } else {
            const float poly = fmaf(u, fmaf(u, 1.0f / 3.0f, 1.0f), 1.0f);
            return poly * e;
        }
    }
}

}  // namespace gpk
