// Rolling prune (§III-A, "Prune-only kernel"): outer list at rlist ->
// inner list at r_inner, with atom-pair in-range masks.
//
// One warp per i-cluster (work counter). For each outer entry the 32 lanes
// test its 64 atom pairs (lane l: pairs (l>>3, l&7) and (l>>3 + 4, l&7),
// i.e. mask bits l and 32 + l) with the FP32 distance contract; the two
// ballots are the new mask words. Entries with an empty mask are dropped.
// The inner list of ci is written at the same offset as its outer list.
#include "nb_internal.cuh"

namespace {

constexpr int kPruneThreads = 256;

struct PruneParams {
    const float4 *xq;
    const int4 *outer;
    int4 *inner;
    const int *ci_start;
    const int *ci_len_outer;
    int *ci_len_inner;
    nb_dev_state *st;
    float Lx, Ly, Lz;
    float r2cut;
    float stale_search2;
};

template <bool SHIFT>
__device__ __forceinline__ bool in_range(const float4 xi, const float4 xj, float Sx, float Sy, float Sz,
                                         float r2cut) {
    float dx = __fsub_rn(xi.x, xj.x), dy = __fsub_rn(xi.y, xj.y), dz = __fsub_rn(xi.z, xj.z);
    if (SHIFT) {
        dx = __fadd_rn(dx, Sx);
        dy = __fadd_rn(dy, Sy);
        dz = __fadd_rn(dz, Sz);
    }
    return nb_r2(dx, dy, dz) < r2cut;
}

__global__ void __launch_bounds__(kPruneThreads) k_prune(PruneParams p) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // displacement since the search must leave the outer list complete at r_inner
        const unsigned ds = p.st->cur_d2_search;
        p.st->last_d2_search = ds;
        p.st->last_d2_prune = 0u;
        p.st->cur_d2_search = 0u;
        p.st->cur_d2_prune = 0u;
        if (__uint_as_float(ds) > p.stale_search2) atomicOr(&p.st->err, NB_DEV_STALE_SEARCH);
    }
    const int lane = threadIdx.x & 31;
    const int b = lane & 7, a1 = lane >> 3, a2 = a1 + 4;
    const unsigned lanebit = 1u << lane;
    const int nc = p.st->nc;
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&p.st->work_prune, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= (unsigned)nc) break;
        const int ci = (int)w;
        const int k0 = p.ci_start[ci], n = p.ci_len_outer[ci];
        const float4 xi1 = p.xq[ci * NB_CLUSTER + a1], xi2 = p.xq[ci * NB_CLUSTER + a2];
        int out = 0;
        for (int k = k0; k < k0 + n; ++k) {
            const int4 e = p.outer[k];
            const float4 xj = p.xq[e.x * NB_CLUSTER + b];
            bool in1, in2;
            if (e.y == NB_SHIFT_CENTER) {
                in1 = in_range<false>(xi1, xj, 0.f, 0.f, 0.f, p.r2cut);
                in2 = in_range<false>(xi2, xj, 0.f, 0.f, 0.f, p.r2cut);
            } else {
                const float Sx = (float)nb_shift_x(e.y) * p.Lx;
                const float Sy = (float)nb_shift_y(e.y) * p.Ly;
                const float Sz = (float)nb_shift_z(e.y) * p.Lz;
                in1 = in_range<true>(xi1, xj, Sx, Sy, Sz, p.r2cut);
                in2 = in_range<true>(xi2, xj, Sx, Sy, Sz, p.r2cut);
            }
            in1 = in1 && ((unsigned)e.z & lanebit);
            in2 = in2 && ((unsigned)e.w & lanebit);
            const unsigned lo = __ballot_sync(0xffffffffu, in1);
            const unsigned hi = __ballot_sync(0xffffffffu, in2);
            if ((lo | hi) != 0u) {
                if (lane == 0) p.inner[k0 + out] = make_int4(e.x, e.y, (int)lo, (int)hi);
                ++out;
            }
        }
        if (lane == 0) {
            p.ci_len_inner[ci] = out;
            atomicAdd(&p.st->inner_count, (unsigned long long)out);
        }
    }
}

}  // namespace

cudaError_t nb_launch_prune(nb_pairlist *pl, float r_inner2, float stale_search2, cudaStream_t s) {
    PruneParams p;
    p.xq = pl->xq;
    p.outer = pl->outer;
    p.inner = pl->inner;
    p.ci_start = pl->ci_start;
    p.ci_len_outer = pl->ci_len_outer;
    p.ci_len_inner = pl->ci_len_inner;
    p.st = pl->st;
    p.Lx = pl->box[0];
    p.Ly = pl->box[1];
    p.Lz = pl->box[2];
    p.r2cut = r_inner2;
    p.stale_search2 = stale_search2;
    // work_prune and inner_count were reset by the snapshot gather before this launch
    int blocks = pl->num_sms * 4;
    blocks = min(blocks, (pl->nc_max + kPruneThreads / 32 - 1) / (kPruneThreads / 32));
    k_prune<<<max(blocks, 1), kPruneThreads, 0, s>>>(p);
    return cudaGetLastError();
}
