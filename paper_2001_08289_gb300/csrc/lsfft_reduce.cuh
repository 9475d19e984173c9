// Deterministic FP64 warp reductions shared by the passes and the finalize step.
#pragma once

#include <cuda_runtime.h>

namespace lsfft {

__host__ __device__ constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : 2 * pow2_at_least((n + 1) / 2); }

// Warp sums of NV values per lane by a reduce-scatter butterfly: with P = NV
// rounded up to a power of two (P <= 32), the step with lane distance o keeps,
// on each lane, the half of its current values selected by the lane's bit o and
// adds the partner lane's copy of that half; after log2 P halving steps the
// remaining distances add single values.  That is P - 1 + 5 - log2 P additions
// instead of 5 NV (this GPU's FP64 pipe makes that count the cost), in an order
// fixed by the lane, so the result is deterministic.  Returns the warp's total
// of value `idx`; lanes whose bits below 32 / P are zero hold distinct indices,
// covering 0..P-1.
template <int NV>
__device__ __forceinline__ double warp_sum_scatter(const double (&acc)[NV], int& idx) {
    constexpr int P = pow2_at_least(NV);
    static_assert(P <= 32, "at most 32 values");
    const int lane = threadIdx.x & 31;
    double v[P];
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = i < NV ? acc[i] : 0.0;
    int base = 0;
#pragma unroll
    for (int h = P / 2, o = 16; h >= 1; h /= 2, o /= 2) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? v[i] : v[i + h];
            const double keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        if (up) base += h;
    }
#pragma unroll
    for (int o = 16 / P; o >= 1; o /= 2) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    idx = base;
    return v[0];
}

}  // namespace lsfft
