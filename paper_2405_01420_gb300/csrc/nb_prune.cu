// Rolling prune (§III-A, "Prune-only kernel"): outer list at rlist ->
// inner list at r_inner, with atom-pair in-range masks.
//
// One warp per i-cluster (work counter). For each outer entry the 32 lanes
// test its 64 atom pairs (lane l: pairs (l>>3, l&7) and (l>>3 + 4, l&7),
// i.e. mask bits l and 32 + l) with the FP32 distance contract; the two
// ballots are the new mask words. Entries with an empty mask are dropped.
// The inner list of ci is written to its own buffer at the same offset as
// its outer list (the kept entries fill a prefix of that range).
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
    const float4 *sys_shift;  // [27 nsys]
    const int *clus_sys;
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

// Tests the 64 atom pairs of one entry; returns the two new mask words.
__device__ __forceinline__ uint2 prune_entry(const int4 e, const float4 xi1, const float4 xi2, const float4 xj,
                                             const unsigned lanebit, const float4 *shift, const PruneParams &p) {
    bool in1, in2;
    if (e.y == NB_SHIFT_CENTER) {
        in1 = in_range<false>(xi1, xj, 0.f, 0.f, 0.f, p.r2cut);
        in2 = in_range<false>(xi2, xj, 0.f, 0.f, 0.f, p.r2cut);
    } else {
        const float4 S = shift[e.y];
        in1 = in_range<true>(xi1, xj, S.x, S.y, S.z, p.r2cut);
        in2 = in_range<true>(xi2, xj, S.x, S.y, S.z, p.r2cut);
    }
    in1 = in1 && ((unsigned)e.z & lanebit);
    in2 = in2 && ((unsigned)e.w & lanebit);
    return make_uint2(__ballot_sync(0xffffffffu, in1), __ballot_sync(0xffffffffu, in2));
}

// One warp per i-cluster. The outer entries of ci are read 32 at a time
// (one per lane, coalesced) into shared memory; the warp tests them two per
// iteration (independent loads for latency hiding); lane t keeps the new
// masks of entry t, and the kept entries are written back compacted and
// coalesced.
__global__ void __launch_bounds__(kPruneThreads) k_prune(PruneParams p) {
    __shared__ int4 s_ent[kPruneThreads / 32][32];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // displacement since the search must leave the outer list complete at r_inner
        const unsigned ds = p.st->cur_d2_search;
        p.st->last_d2_search = ds;
        p.st->last_d2_prune = 0u;
        p.st->cur_d2_search = 0u;
        p.st->cur_d2_prune = 0u;
        if (__uint_as_float(ds) > p.stale_search2) atomicOr(&p.st->err, NB_DEV_STALE_SEARCH);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = lane & 7, a1 = lane >> 3, a2 = a1 + 4;
    const unsigned lanebit = 1u << lane;
    int4 *ent = s_ent[warp];
    const int nc = p.st->nc;
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&p.st->work_prune, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= (unsigned)nc) break;
        const int ci = (int)w;
        const float4 *shift = p.sys_shift + 27 * p.clus_sys[ci];
        const int k0 = p.ci_start[ci], n = p.ci_len_outer[ci];
        const float4 xi1 = p.xq[ci * NB_CLUSTER + a1], xi2 = p.xq[ci * NB_CLUSTER + a2];
        int out = 0;
        for (int base = 0; base < n; base += 32) {
            const int cnt = min(32, n - base);
            __syncwarp();
            if (lane < cnt) ent[lane] = p.outer[k0 + base + lane];
            __syncwarp();
            uint2 mine = make_uint2(0u, 0u);
            int t = 0;
            for (; t + 1 < cnt; t += 2) {
                const int4 e0 = ent[t], e1 = ent[t + 1];
                const float4 xj0 = p.xq[e0.x * NB_CLUSTER + b];
                const float4 xj1 = p.xq[e1.x * NB_CLUSTER + b];
                const uint2 m0 = prune_entry(e0, xi1, xi2, xj0, lanebit, shift, p);
                const uint2 m1 = prune_entry(e1, xi1, xi2, xj1, lanebit, shift, p);
                if (lane == t) mine = m0;
                if (lane == t + 1) mine = m1;
            }
            if (t < cnt) {
                const int4 e0 = ent[t];
                const uint2 m0 = prune_entry(e0, xi1, xi2, p.xq[e0.x * NB_CLUSTER + b], lanebit, shift, p);
                if (lane == t) mine = m0;
            }
            const bool keep = lane < cnt && (mine.x | mine.y) != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int4 e = ent[lane];
                p.inner[k0 + out + __popc(bal & (lanebit - 1u))] = make_int4(e.x, e.y, (int)mine.x, (int)mine.y);
            }
            out += __popc(bal);
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
    p.sys_shift = pl->sys_shift;
    p.clus_sys = pl->clus_sys;
    p.r2cut = r_inner2;
    p.stale_search2 = stale_search2;
    // work_prune and inner_count were reset by the snapshot gather before this launch
    int blocks = pl->num_sms * 4;
    blocks = min(blocks, (pl->nc_max + kPruneThreads / 32 - 1) / (kPruneThreads / 32));
    k_prune<<<max(blocks, 1), kPruneThreads, 0, s>>>(p);
    return cudaGetLastError();
}
