// Smooth particle-mesh Ewald charge spreading and force gathering, B-spline
// order 4 (the long-range part that §III-A places next to the short-range
// kernel; Essmann et al. 1995 define it). Declared in include/nb.h.
//
// Both kernels give each atom 4 lanes: lane c owns the z point base_z - c
// of the atom's 4 x 4 x 4 support and walks its 16 (x, y) points itself.
// A warp instruction then touches 8 atoms x 4 consecutive floats (one
// 16-byte run per atom), and each atom's x and y spline weights are
// computed 4 times rather than 16.
// The kernels are bound by instruction issue more than by the L2 (16 lanes
// per atom, each recomputing every weight, issued 2 to 4 times as many
// instructions for the same atomics and loads).
//
// Scaled coordinates. u = x K / L has |u| up to K (about 100): in plain
// FP32 its fractional part, which the weights depend on, would carry an
// error of K 2^-24 (6e-6). Here K / L comes in as an unevaluated FP32 pair
// (hi + lo) and the product x (hi + lo) is formed exactly up to the last
// term (fma gives x hi's rounding error), so the fractional part is right
// to about 2^-24 absolute whatever K is.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "nb_internal.cuh"

namespace {

constexpr int kOrder = 4;
constexpr int kThreads = 256;
constexpr int kLanesPerAtom = 4;

struct pme_axes {
    float s_hi[3], s_lo[3];  // K_a / L_a as hi + lo
    float s[3];              // K_a / L_a rounded (the force's chain-rule factor)
    float Kf[3], invK[3];    // K_a and 1 / K_a rounded
    int K[3];
};

// Fractional part w in [0, 1) and mesh index base in [0, K) of u = x K / L.
// The index is reduced modulo K in FP32 (exact for |floor(u)| < 2^24) instead
// of an integer division; anything else (huge or non-finite coordinates)
// ends at index 0, never outside the mesh.
__device__ __forceinline__ void pme_scaled(float x, float s_hi, float s_lo, float Kf, float invK, int K, float &w,
                                           int &base) {
    const float t = __fmul_rn(x, s_hi);
    const float e = __fmaf_rn(x, s_hi, -t);        // exact rounding error of t
    const float lo = __fmaf_rn(x, s_lo, e);        // the rest of the product
    float fl = floorf(t);
    float f = __fadd_rn(__fsub_rn(t, fl), lo);     // t - fl is exact
    if (f < 0.0f) { f = __fadd_rn(f, 1.0f); fl = __fsub_rn(fl, 1.0f); }
    if (f >= 1.0f) { f = __fsub_rn(f, 1.0f); fl = __fadd_rn(fl, 1.0f); }
    if (f >= 1.0f) f = 0x1.fffffep-1f;             // 1 - 2^-24 rounded up to 1
    w = f;
    int b = (int)__fmaf_rn(-Kf, floorf(__fmul_rn(fl, invK)), fl);  // fl - K floor(fl / K)
    if (b < 0) b += K;
    if (b >= K) b -= K;
    base = (unsigned)b < (unsigned)K ? b : 0;
}

// Cubic B-spline weights of mesh points base - j, M4(w + j) for j = 0..3,
// by the closed form of the uniform cubic B-spline:
//   M4(w) = w^3/6,  M4(w+1) = (-3w^3 + 3w^2 + 3w + 1)/6,
//   M4(w+2) = (3w^3 - 6w^2 + 4)/6,  M4(w+3) = (1 - w)^3/6.
__device__ __forceinline__ void pme_w4(float w, float m[4]) {
    const float v = 1.0f - w;
    const float w2 = w * w, w3 = w2 * w;
    m[0] = w3 * (1.0f / 6.0f);
    m[3] = v * v * v * (1.0f / 6.0f);
    m[1] = __fmaf_rn(-3.0f, w3, __fmaf_rn(3.0f, w2, __fmaf_rn(3.0f, w, 1.0f))) * (1.0f / 6.0f);
    m[2] = __fmaf_rn(3.0f, w3, __fmaf_rn(-6.0f, w2, 4.0f)) * (1.0f / 6.0f);
}

// dM4/du at w + j: w^2/2, (-3w^2 + 2w + 1)/2, (3w^2 - 4w)/2, -(1 - w)^2/2
__device__ __forceinline__ void pme_d4(float w, float d[4]) {
    const float v = 1.0f - w;
    const float w2 = w * w;
    d[0] = 0.5f * w2;
    d[1] = 0.5f * __fmaf_rn(-3.0f, w2, __fmaf_rn(2.0f, w, 1.0f));
    d[2] = 0.5f * __fmaf_rn(3.0f, w2, -4.0f * w);
    d[3] = -0.5f * v * v;
}

__device__ __forceinline__ float pme_pick(const float m[4], int j) {
    return j == 0 ? m[0] : j == 1 ? m[1] : j == 2 ? m[2] : m[3];
}

// Mesh offsets of an atom's support, per lane: x planes (times K1 K2) and
// y rows (times K2) for j = 0..3, and the lane's own z point.
__device__ __forceinline__ void pme_offsets(const pme_axes &ax, const int base[3], int c, int xo[4], int yo[4],
                                            int &zc) {
    const int plane = ax.K[1] * ax.K[2];
#pragma unroll
    for (int j = 0; j < kOrder; ++j) {
        int ix = base[0] - j, iy = base[1] - j;
        if (ix < 0) ix += ax.K[0];
        if (iy < 0) iy += ax.K[1];
        xo[j] = ix * plane;
        yo[j] = iy * ax.K[2];
    }
    zc = base[2] - c;
    if (zc < 0) zc += ax.K[2];
}

__global__ void __launch_bounds__(kThreads) k_pme_spread(int n, const float *__restrict__ coords,
                                                         const float *__restrict__ q, pme_axes ax,
                                                         float *__restrict__ grid) {
    const int c = threadIdx.x & (kLanesPerAtom - 1);
    // unsigned: n < 2^31 and the stride is below 2^17, so i + stride never wraps
    const unsigned stride = gridDim.x * (kThreads / kLanesPerAtom);
    for (unsigned i = blockIdx.x * (kThreads / kLanesPerAtom) + (threadIdx.x >> 2); i < (unsigned)n; i += stride) {
        const float qi = __ldg(q + i);
        const float *xi = coords + 3 * (size_t)i;
        float w[3];
        int base[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            pme_scaled(__ldg(xi + a), ax.s_hi[a], ax.s_lo[a], ax.Kf[a], ax.invK[a], ax.K[a], w[a],
                       base[a]);
        float mx[4], my[4], mz[4];
        pme_w4(w[0], mx);
        pme_w4(w[1], my);
        pme_w4(w[2], mz);
        const float v = qi * pme_pick(mz, c);
        int xo[4], yo[4], zc;
        pme_offsets(ax, base, c, xo, yo, zc);
#pragma unroll
        for (int a = 0; a < kOrder; ++a) {
            const float va = v * mx[a];
#pragma unroll
            for (int b = 0; b < kOrder; ++b) atomicAdd(grid + (xo[a] + yo[b] + zc), va * my[b]);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_pme_gather(int n, const float *__restrict__ coords,
                                                         const float *__restrict__ q, pme_axes ax,
                                                         const float *__restrict__ phi, float *__restrict__ forces,
                                                         int accumulate, double *__restrict__ energy) {
    const int c = threadIdx.x & (kLanesPerAtom - 1);
    const long long stride = (long long)gridDim.x * (kThreads / kLanesPerAtom);
    double e_acc = 0.0;
    // every lane group runs the same number of iterations, so the shuffles below see all 32 lanes
    const long long n_round = ((long long)n + stride - 1) / stride * stride;
    for (long long i = (long long)blockIdx.x * (kThreads / kLanesPerAtom) + (threadIdx.x >> 2); i < n_round;
         i += stride) {
        const bool live = i < n;
        float psi = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f, qi = 0.0f;
        if (live) {
            qi = __ldg(q + i);
            float w[3];
            int base[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                pme_scaled(__ldg(coords + 3 * i + a), ax.s_hi[a], ax.s_lo[a], ax.Kf[a], ax.invK[a], ax.K[a], w[a],
                           base[a]);
            float mx[4], dx[4], my[4], dy[4];
            pme_w4(w[0], mx);
            pme_d4(w[0], dx);
            pme_w4(w[1], my);
            pme_d4(w[1], dy);
            int xo[4], yo[4], zc;
            pme_offsets(ax, base, c, xo, yo, zc);
            float p[kOrder][kOrder];
#pragma unroll
            for (int a = 0; a < kOrder; ++a)
#pragma unroll
                for (int b = 0; b < kOrder; ++b) p[a][b] = __ldg(phi + (xo[a] + yo[b] + zc));
            float s_m = 0.0f, s_dx = 0.0f, s_dy = 0.0f;  // sums over the lane's 16 (x, y) points
#pragma unroll
            for (int a = 0; a < kOrder; ++a) {
                float sm = 0.0f, sd = 0.0f;  // sum_b M(y_b) phi, sum_b M'(y_b) phi on plane a
#pragma unroll
                for (int b = 0; b < kOrder; ++b) {
                    sm = __fmaf_rn(my[b], p[a][b], sm);
                    sd = __fmaf_rn(dy[b], p[a][b], sd);
                }
                s_m = __fmaf_rn(mx[a], sm, s_m);
                s_dx = __fmaf_rn(dx[a], sm, s_dx);
                s_dy = __fmaf_rn(mx[a], sd, s_dy);
            }
            float mz4[4], dz4[4];
            pme_w4(w[2], mz4);
            pme_d4(w[2], dz4);
            const float mz = pme_pick(mz4, c), dz = pme_pick(dz4, c);
            psi = mz * s_m;
            gx = mz * s_dx;
            gy = mz * s_dy;
            gz = dz * s_m;
        }
#pragma unroll
        for (int o = 1; o < kLanesPerAtom; o <<= 1) {
            psi += __shfl_xor_sync(0xffffffffu, psi, o);
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if (live && c == 0) {
            const float f[3] = {-qi * ax.s[0] * gx, -qi * ax.s[1] * gy, -qi * ax.s[2] * gz};
#pragma unroll
            for (int a = 0; a < 3; ++a) forces[3 * i + a] = accumulate ? forces[3 * i + a] + f[a] : f[a];
            e_acc += 0.5 * (double)qi * (double)psi;
        }
    }
    if (energy) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
        if ((threadIdx.x & 31) == 0 && e_acc != 0.0) atomicAdd(energy, e_acc);
    }
}

int pme_check(const char *who, int n, const float *coords, const float *q, const float *box, int K0, int K1, int K2,
              int order, pme_axes &ax) {
    char msg[160];
    if (n < 0) {
        snprintf(msg, sizeof msg, "%s: n_atoms < 0", who);
        return nb_record_error(NB_ERR_ARG, msg);
    }
    if ((n > 0 && (!coords || !q)) || !box) {
        snprintf(msg, sizeof msg, "%s: NULL argument", who);
        return nb_record_error(NB_ERR_ARG, msg);
    }
    if (order != kOrder) {
        snprintf(msg, sizeof msg, "%s: only B-spline order 4 is built", who);
        return nb_record_error(NB_ERR_ARG, msg);
    }
    const int K[3] = {K0, K1, K2};
    if ((long long)K0 * K1 * K2 > 2147483647LL) {
        snprintf(msg, sizeof msg, "%s: the mesh must have fewer than 2^31 points", who);
        return nb_record_error(NB_ERR_ARG, msg);
    }
    for (int a = 0; a < 3; ++a) {
        if (K[a] < kOrder || K[a] > 4096) {
            snprintf(msg, sizeof msg, "%s: each mesh dimension must be in [4, 4096]", who);
            return nb_record_error(NB_ERR_ARG, msg);
        }
        if (!(box[a] > 0.0f) || !(box[a] < 1e30f)) {
            snprintf(msg, sizeof msg, "%s: each box edge must be positive and finite", who);
            return nb_record_error(NB_ERR_ARG, msg);
        }
        const double s = (double)K[a] / (double)box[a];
        ax.K[a] = K[a];
        ax.Kf[a] = (float)K[a];
        ax.invK[a] = (float)(1.0 / K[a]);
        ax.s[a] = (float)s;
        ax.s_hi[a] = (float)s;
        ax.s_lo[a] = (float)(s - (double)ax.s_hi[a]);
    }
    return NB_OK;
}

// One wave of resident blocks (the kernels stride over the atoms), or fewer
// for a small system. The SM count and the kernel's occupancy are looked up
// once per device and kernel (kind 0 spread, 1 gather).
constexpr int kMaxDevices = 64;
int g_pme_sms[kMaxDevices] = {};
int g_pme_per_sm[kMaxDevices][2] = {};

int pme_blocks(int n, const void *kernel, int kind) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    if (g_pme_sms[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        g_pme_sms[dev] = sms;
    }
    if (g_pme_per_sm[dev][kind] == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        g_pme_per_sm[dev][kind] = per_sm;
    }
    const long long want = ((long long)n * kLanesPerAtom + kThreads - 1) / kThreads;
    return (int)std::max(1LL, std::min(want, (long long)g_pme_sms[dev] * g_pme_per_sm[dev][kind]));
}

}  // namespace

extern "C" int nb_pme_spread(int n_atoms, const float *coords, const float *q, const float *box, int K0, int K1, int K2,
                             int order, float *grid, void *stream) {
    pme_axes ax;
    int rc = pme_check("nb_pme_spread", n_atoms, coords, q, box, K0, K1, K2, order, ax);
    if (rc != NB_OK) return rc;
    if (!grid) return nb_record_error(NB_ERR_ARG, "nb_pme_spread: NULL grid");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cells = (size_t)K0 * K1 * K2;
    cudaError_t e = cudaMemsetAsync(grid, 0, sizeof(float) * cells, s);
    if (e == cudaSuccess && n_atoms > 0) {
        k_pme_spread<<<pme_blocks(n_atoms, (const void *)k_pme_spread, 0), kThreads, 0, s>>>(n_atoms, coords, q, ax, grid);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nb_record_error(NB_ERR_CUDA, cudaGetErrorString(e));
    return NB_OK;
}

extern "C" int nb_pme_gather(int n_atoms, const float *coords, const float *q, const float *box, int K0, int K1, int K2,
                             int order, const float *phi, float *forces, int accumulate, double *energy,
                             void *stream) {
    pme_axes ax;
    int rc = pme_check("nb_pme_gather", n_atoms, coords, q, box, K0, K1, K2, order, ax);
    if (rc != NB_OK) return rc;
    if (!phi || (n_atoms > 0 && !forces)) return nb_record_error(NB_ERR_ARG, "nb_pme_gather: NULL phi or forces");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (energy) e = cudaMemsetAsync(energy, 0, sizeof(double), s);
    if (e == cudaSuccess && n_atoms > 0) {
        k_pme_gather<<<pme_blocks(n_atoms, (const void *)k_pme_gather, 1), kThreads, 0, s>>>(
            n_atoms, coords, q, ax, phi, forces, accumulate ? 1 : 0, energy);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nb_record_error(NB_ERR_CUDA, cudaGetErrorString(e));
    return NB_OK;
}
