// Warp-level helpers of the gathered-tile kernels: asynchronous copies into
// shared memory and a reduce-scatter of per-lane partial sums.
#pragma once

#include <cuda_runtime.h>

// cp.async of 16 / 4 bytes, global -> shared (cached in L1).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem) : "memory");
}

// cp.async of 4 bytes of which the first n (0 or 4) are read from gmem and
// the rest are zero-filled; with n = 0 nothing is read.
__device__ __forceinline__ void cp_async4_zfill(void *smem, const void *gmem, unsigned n) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gmem), "r"(n) : "memory");
}

// Waits for this thread's outstanding cp.async copies.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Sums v[0..N-1] (N = 8, 16 or 32) over the 32 lanes of the warp. Each step
// halves the values a lane holds: lanes with bit o set keep the upper half
// and send the lower one to lane ^ o, and the other way round. On return
// v[0] of lane l holds the warp total of value l >> (5 - log2 N).
template <int N>
__device__ __forceinline__ void reduce_scatter(float (&v)[N], int lane) {
    static_assert(N == 8 || N == 16 || N == 32, "reduce_scatter: N must be 8, 16 or 32");
    int o = 16;
#pragma unroll
    for (int n = N; n > 1; n >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float send = upper ? v[i] : v[i + n / 2];
            const float keep = upper ? v[i + n / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}
