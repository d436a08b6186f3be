// Excluded-pair correction (NB_COUL_EXCL_CORR): the excluded atom pairs
// within rc carry
//   Ewald:           e = -f qi qj erf(beta r)/r   (erfc/r - 1/r)
//   reaction field:  e =  f qi qj (k_rf r^2 - c_rf)
// with F_i = -de/dx_i. The pairs come from the exclusion lists given to the
// search: k_excl_list records them there (each pair once, i < j) as slot
// pairs in a buffer the pair list owns, so later calls do not read the
// caller's lists. This is O(number of exclusions), independent of the pair
// list. The positions are the current images y in cluster order (xq,
// written by the gather), the displacement is taken to the minimum image of
// the system's box, and forces go to the same float4 accumulators as the
// pair kernels.
//
// k_excl_list      exclusion lists -> slot pairs (during the search)
// k_excl_corr      forces and the E_coul contribution
// k_excl_corr_adj  its adjoint for g = dL/dF (dL/dx, dL/dq)
//
// Per pair (per unit f qi qj) B = -(1/r) de/dr and D = (1/r) dB/dr:
//   Ewald: B = [(2 beta/sqrt(pi)) exp(-beta^2 r^2) - erf(beta r)/r] / r^2,
//          D = [-3 B - 2 (2 beta/sqrt(pi)) beta^2 exp(-beta^2 r^2)] / r^2
//   RF:    B = -2 k_rf, D = 0.
// erf and exp are CUDA's erff / expf: this kernel is small next to the pair
// kernels.
#include "nb_pair.cuh"

namespace {

constexpr int kExclThreads = 256;

struct ExclParams {
    const int2 *pairs;    // (slot_i, slot_j)
    const nb_dev_state *st;
    unsigned cap;
    const float4 *xq;     // (y, q) per slot
    float4 *acc;          // fsort (forward) or bsort (adjoint) per slot
    const float4 *gsort;  // adjoint: g per slot
    const int *clus_sys;
    const nb_sys *sys;
    double *energies;  // [2 nsys] or NULL
    nb_coul cc;
};

// One thread per atom; the warp reserves the places of its pairs with one
// atomic per round (all threads of a warp on one counter would serialise).
__global__ void __launch_bounds__(kExclThreads) k_excl_list(int n, const int *__restrict__ excl_off,
                                                            const int *__restrict__ excl_idx,
                                                            const int *__restrict__ pos, int2 *__restrict__ pairs,
                                                            unsigned cap, nb_dev_state *st) {
    const int lane = threadIdx.x & 31;
    // every lane of a warp runs the same rounds, so the warp-wide votes below see all of it
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + (int)threadIdx.x;
        int k = i < n ? excl_off[i] : 0;
        const int k1 = i < n ? excl_off[i + 1] : 0;
        for (;;) {
            // this lane's next pair with j > i (each pair once; indices outside [0, n) are flagged by the search)
            int j = -1;
            while (k < k1 && j < 0) {
                const int c = excl_idx[k++];
                if (c > i && c < n) j = c;
            }
            const bool has = j >= 0;
            const unsigned bal = __ballot_sync(0xffffffffu, has);
            if (bal == 0u) break;
            unsigned base = 0u;
            if (lane == __ffs(bal) - 1) base = atomicAdd(&st->excl_count, (unsigned)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
            if (has) {
                const unsigned idx = base + (unsigned)__popc(bal & ((1u << lane) - 1u));
                if (idx < cap)
                    pairs[idx] = make_int2(pos[i], pos[j]);
                else
                    atomicOr(&st->err, NB_DEV_EXCL_OVERFLOW);
            }
        }
    }
}

// Radial terms of an excluded pair at r2 (< rc2, > 0): e + e_lo (per f qi
// qj; e_lo carries the residuals of the RF constants), B, D.
template <bool RF>
__device__ __forceinline__ void excl_radial(const nb_coul &cc, float r2, float &e, float &e_lo, float &B, float &D) {
    e_lo = 0.0f;
    if (RF) {
        e = fmaf(cc.krf, r2, -cc.crf);
        e_lo = fmaf(cc.krf_lo, r2, -cc.crf_lo);
        B = -2.0f * cc.krf;
        D = 0.0f;
    } else {
        const float r = sqrtf(r2), rinv = 1.0f / r, rinv2 = rinv * rinv;
        const float erfv = erff(cc.beta * r);
        const float ex = expf(-cc.beta * cc.beta * r2);
        e = -erfv * rinv;
        B = fmaf(cc.c2b, ex, -erfv * rinv) * rinv2;
        D = fmaf(-3.0f, B, -2.0f * cc.c2b * cc.beta * cc.beta * ex) * rinv2;
    }
}

// Minimum-image displacement y_i - y_j in the system's box.
__device__ __forceinline__ float3 excl_disp(const float4 yi, const float4 yj, const float4 L) {
    float3 d = make_float3(yi.x - yj.x, yi.y - yj.y, yi.z - yj.z);
    d.x -= L.x * rintf(d.x / L.x);
    d.y -= L.y * rintf(d.y / L.y);
    d.z -= L.z * rintf(d.z / L.z);
    return d;
}

// Adds v to the system's E_coul: one atomic per warp when the whole warp is
// in one system (the usual case), one per lane otherwise.
__device__ __forceinline__ void add_energy(double v, int sys, double *energies) {
    const int sys0 = __shfl_sync(0xffffffffu, sys, 0);
    if (__all_sync(0xffffffffu, sys == sys0)) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&energies[2 * sys0 + 1], v);
    } else if (v != 0.0) {
        atomicAdd(&energies[2 * sys + 1], v);
    }
}

template <bool RF>
__global__ void __launch_bounds__(kExclThreads) k_excl_corr(ExclParams p) {
    const unsigned np = min(p.st->excl_count, p.cap);
    const unsigned stride = gridDim.x * blockDim.x;
    // every lane runs the same number of rounds, so the warp-level energy sum is uniform
    for (unsigned base = blockIdx.x * blockDim.x; base < np; base += stride) {
        const unsigned k = base + threadIdx.x;
        double e_sum = 0.0;
        int sys = 0;
        if (k < np) {
            const int2 pr = p.pairs[k];
            sys = p.clus_sys[pr.x / NB_CLUSTER];
            const float4 yi = p.xq[pr.x], yj = p.xq[pr.y];
            const float3 d = excl_disp(yi, yj, p.sys[sys].box);
            const float r2 = fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x));
            if (r2 < p.cc.rc2 && r2 > 0.0f) {
                float e, e_lo, B, D;
                excl_radial<RF>(p.cc, r2, e, e_lo, B, D);
                const float qq = NB_COULOMB_F * yi.w * yj.w;
                const float s = qq * B;
                atomicAdd(p.acc + pr.x, make_float4(s * d.x, s * d.y, s * d.z, 0.0f));
                atomicAdd(p.acc + pr.y, make_float4(-s * d.x, -s * d.y, -s * d.z, 0.0f));
                e_sum = (double)qq * e + (double)qq * e_lo;
            }
        }
        if (p.energies) add_energy(e_sum, sys, p.energies);
    }
}

template <bool RF>
__global__ void __launch_bounds__(kExclThreads) k_excl_corr_adj(ExclParams p) {
    const unsigned np = min(p.st->excl_count, p.cap);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const int2 pr = p.pairs[k];
        const float4 yi = p.xq[pr.x], yj = p.xq[pr.y];
        const float4 gi = p.gsort[pr.x], gj = p.gsort[pr.y];
        const float3 d = excl_disp(yi, yj, p.sys[p.clus_sys[pr.x / NB_CLUSTER]].box);
        const float r2 = fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x));
        if (!(r2 < p.cc.rc2) || !(r2 > 0.0f)) continue;
        float e, e_lo, B, D;
        excl_radial<RF>(p.cc, r2, e, e_lo, B, D);
        const float fqi = NB_COULOMB_F * yi.w, fqj = NB_COULOMB_F * yj.w;
        const float qq = fqi * yj.w;
        const float s = qq * B, spr = qq * D;
        const float ux = gi.x - gj.x, uy = gi.y - gj.y, uz = gi.z - gj.z;
        const float ud = fmaf(ux, d.x, fmaf(uy, d.y, uz * d.z));
        const float t = spr * ud;
        const float vx = fmaf(s, ux, t * d.x), vy = fmaf(s, uy, t * d.y), vz = fmaf(s, uz, t * d.z);
        atomicAdd(p.acc + pr.x, make_float4(vx, vy, vz, fqj * B * ud));
        atomicAdd(p.acc + pr.y, make_float4(-vx, -vy, -vz, fqi * B * ud));
    }
}

ExclParams make_params(nb_pairlist *pl, float rc, float beta, bool &rf) {
    ExclParams p;
    p.pairs = pl->excl_pairs;
    p.st = pl->st;
    p.cap = (unsigned)pl->excl_cap;
    p.xq = pl->xq;
    p.gsort = pl->gsort;
    p.clus_sys = pl->clus_sys;
    p.sys = pl->sys;
    p.energies = nullptr;
    rf = nb_fill_coul(p.cc, rc, beta, pl->coul_kind, pl->eps_rf, pl->coul_flags) == NB_COULK_RF;
    return p;
}

int excl_blocks(const nb_pairlist *pl) {
    return max(1, min((int)((pl->excl_cap + kExclThreads - 1) / kExclThreads), pl->num_sms * 8));
}

}  // namespace

cudaError_t nb_launch_excl_list(nb_pairlist *pl, const int *excl_off, const int *excl_idx, cudaStream_t s) {
    const int blocks = max(1, min((pl->n_atoms + kExclThreads - 1) / kExclThreads, pl->num_sms * 8));
    k_excl_list<<<blocks, kExclThreads, 0, s>>>(pl->n_atoms, excl_off, excl_idx, pl->pos, pl->excl_pairs,
                                                 (unsigned)pl->excl_cap, pl->st);
    return cudaGetLastError();
}

cudaError_t nb_launch_excl_corr(nb_pairlist *pl, float rc, float beta, double *energies, cudaStream_t s) {
    bool rf;
    ExclParams p = make_params(pl, rc, beta, rf);
    p.acc = pl->fsort;
    p.energies = energies;
    if (rf)
        k_excl_corr<true><<<excl_blocks(pl), kExclThreads, 0, s>>>(p);
    else
        k_excl_corr<false><<<excl_blocks(pl), kExclThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t nb_launch_excl_corr_adj(nb_pairlist *pl, float rc, float beta, cudaStream_t s) {
    bool rf;
    ExclParams p = make_params(pl, rc, beta, rf);
    p.acc = pl->bsort;
    if (rf)
        k_excl_corr_adj<true><<<excl_blocks(pl), kExclThreads, 0, s>>>(p);
    else
        k_excl_corr_adj<false><<<excl_blocks(pl), kExclThreads, 0, s>>>(p);
    return cudaGetLastError();
}
