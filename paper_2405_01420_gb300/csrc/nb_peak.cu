// nb_fp32_peak_probe: the FP32 throughput the force kernel's roofline divides
// by, measured rather than taken from unit counts. Declared in include/nb.h.
//
// Every thread runs NB_PEAK_CHAINS independent fused multiply-add chains,
// x <- fma(x, a, b), so the FMA pipe always has independent work and the
// chains' latency is hidden by their number, not by other instructions. The
// scalar form issues one FFMA per fused multiply-add; the packed form issues
// one two-wide FFMA2 (__ffma2_rn) for two of them, as the force kernel's row
// pairs do. The loop's own instructions (a counter and a branch per 128 or
// 256 fused multiply-adds) are below 1% of the issue slots.
#include "nb_internal.cuh"

namespace {

constexpr int kChains = 8;    // independent chains per thread (per lane of a packed pair)
constexpr int kUnroll = 16;   // chain steps per loop iteration
constexpr int kThreads = 256;

template <bool PACKED>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, float a, float b, float *out) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (PACKED) {
        float2 x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = make_float2(1e-3f * (float)(tid & 255) + c, 0.5f * c);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
        }
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
        out[tid] = s;
    } else {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(tid & 255) + c;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
        }
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c];
        out[tid] = s;
    }
}

}  // namespace

extern "C" int nb_fp32_peak_probe(int packed, int blocks_per_sm, int iters, float *out, size_t out_len,
                                  double *flops, void *stream) {
    if (!out || !flops) return nb_record_error(NB_ERR_ARG, "nb_fp32_peak_probe: NULL argument");
    if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8)
        return nb_record_error(NB_ERR_ARG, "nb_fp32_peak_probe: need iters >= 1 and 1 <= blocks_per_sm <= 8");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return nb_record_error(NB_ERR_CUDA, "nb_fp32_peak_probe: no usable current device");
    const size_t threads = (size_t)sms * blocks_per_sm * kThreads;
    if (out_len < threads)
        return nb_record_error(NB_ERR_ARG, "nb_fp32_peak_probe: out holds fewer floats than the grid has threads");
    cudaStream_t s = (cudaStream_t)stream;
    // a = 1 - 2^-20 and b = 2^-20 keep every chain near 1: no overflow, no subnormals
    const float a = 1.0f - 0x1p-20f, b = 0x1p-20f;
    if (packed)
        k_fma_probe<true><<<sms * blocks_per_sm, kThreads, 0, s>>>(iters, a, b, out);
    else
        k_fma_probe<false><<<sms * blocks_per_sm, kThreads, 0, s>>>(iters, a, b, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nb_record_error(NB_ERR_CUDA, cudaGetErrorString(e));
    *flops = 2.0 * (packed ? 2.0 : 1.0) * (double)threads * iters * kUnroll * kChains;
    return NB_OK;
}
