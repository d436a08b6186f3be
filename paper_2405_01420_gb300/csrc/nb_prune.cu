// Rolling prune (§III-A, "Prune-only kernel"): outer list at rlist ->
// inner list at r_inner, with atom-pair in-range masks. As in the paper's
// post-pruning list sorting, the prune also computes the list-size
// histogram that the sort needs.
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
    int *vt_slot;        // [2 cap * 8] gathered j slots (shift index in the top 5 bits)
    unsigned *vt_mask;   // [2 cap] 4 x 8 in-range bits (bit a*8 + p)
    int *half_start;     // [2 nc_max]
    int *half_len;       // [2 nc_max]
    int pad_slot;        // a slot that never holds an atom (far away, q = 0)
    int *len_key;        // [nc_max] work of each i-cluster for the force kernel
    int *len_hist;       // [NB_LEN_BINS] histogram of len_key, or NULL (no sorting)
    float r2cut;
    float stale_search2;
};

constexpr int kStage = 512;  // ring of staged j atoms per warp and half (>= 32 * 8 + 8)

// Rows (a = 0..3) of column b of a 4 x 8 mask (bit a*8 + b) as 4 bits.
__device__ __forceinline__ unsigned column_rows(unsigned m, int b) {
    return ((m >> b) & 1u) | ((m >> (7 + b)) & 2u) | ((m >> (14 + b)) & 4u) | ((m >> (21 + b)) & 8u);
}

// Writes one gathered tile from the 8 staged atoms at ring position head.
__device__ __forceinline__ void flush_tile(const int *ring_slot, const unsigned char *ring_rows, int head, int vt,
                                           int lane, const PruneParams &p) {
    const int idx = (head + (lane & 7)) & (kStage - 1);
    const int v = ring_slot[idx];
    const unsigned r = lane < 8 ? ring_rows[idx] : 0u;
    if (lane < 8) p.vt_slot[8 * (size_t)vt + lane] = v;
    unsigned m = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) m |= (__ballot_sync(0xffffffffu, (r >> a) & 1u) & 0xffu) << (8 * a);
    if (lane == 0) p.vt_mask[vt] = m;
}

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
template <bool TILES>
__global__ void __launch_bounds__(kPruneThreads) k_prune(PruneParams p) {
    __shared__ int4 s_ent[kPruneThreads / 32][32];
    __shared__ int s_rslot[kPruneThreads / 32][2][kStage];
    __shared__ unsigned char s_rrows[kPruneThreads / 32][2][kStage];
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
        // tiles of half h go to [2 k0 + h n, 2 k0 + (h + 1) n): each entry adds at most 8 atoms
        const float4 xi1 = p.xq[ci * NB_CLUSTER + a1], xi2 = p.xq[ci * NB_CLUSTER + a2];
        int out = 0;
        int head[2] = {0, 0}, fill[2] = {0, 0}, ntile[2] = {0, 0};
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
            const int4 e = ent[lane];
            if (keep)
                p.inner[k0 + out + __popc(bal & (lanebit - 1u))] = make_int4(e.x, e.y, (int)mine.x, (int)mine.y);
            out += __popc(bal);
            // Gather, per half, the j atoms in range of any of its 4 rows.
#pragma unroll
            for (int h = 0; h < (TILES ? 2 : 0); ++h) {
                const unsigned m = lane < cnt ? (h ? mine.y : mine.x) : 0u;
                unsigned col = (m | (m >> 8) | (m >> 16) | (m >> 24)) & 0xffu;
                const int c = __popc(col);
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                int pos = head[h] + fill[h] + incl - c;
                while (col) {
                    const int bb = __ffs(col) - 1;
                    col &= col - 1u;
                    const int idx = pos & (kStage - 1);
                    s_rslot[warp][h][idx] = (int)((unsigned)(e.x * NB_CLUSTER + bb) | ((unsigned)e.y << 27));
                    s_rrows[warp][h][idx] = (unsigned char)column_rows(m, bb);
                    ++pos;
                }
                fill[h] += total;
                __syncwarp();
                while (fill[h] >= 8) {
                    flush_tile(s_rslot[warp][h], s_rrows[warp][h], head[h], 2 * k0 + h * n + ntile[h], lane, p);
                    head[h] += 8;
                    fill[h] -= 8;
                    ++ntile[h];
                }
                __syncwarp();
            }
        }
        // last partial tile of each half, padded with a slot that holds no atom
#pragma unroll
        for (int h = 0; h < (TILES ? 2 : 0); ++h) {
            if (fill[h] > 0) {
                if (lane >= fill[h] && lane < 8) {
                    const int idx = (head[h] + lane) & (kStage - 1);
                    s_rslot[warp][h][idx] = (int)((unsigned)p.pad_slot | ((unsigned)NB_SHIFT_CENTER << 27));
                    s_rrows[warp][h][idx] = 0;
                }
                __syncwarp();
                flush_tile(s_rslot[warp][h], s_rrows[warp][h], head[h], 2 * k0 + h * n + ntile[h], lane, p);
                ++ntile[h];
            }
            if (lane == 0) {
                p.half_start[2 * ci + h] = 2 * k0 + h * n;
                p.half_len[2 * ci + h] = ntile[h];
            }
        }
        __syncwarp();
        if (lane == 0) {
            p.ci_len_inner[ci] = out;
            atomicAdd(&p.st->inner_count, (unsigned long long)out);
            // post-prune sorting: the force kernel's work for ci and its histogram
            const int key = TILES ? ntile[0] + ntile[1] : out;
            p.len_key[ci] = key;
            if (p.len_hist) atomicAdd(&p.len_hist[min(key, NB_LEN_BINS - 1)], 1);
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
    p.vt_slot = pl->vt_slot;
    p.vt_mask = pl->vt_mask;
    p.half_start = pl->half_start;
    p.half_len = pl->half_len;
    p.pad_slot = pl->nc_max * NB_CLUSTER;
    p.len_key = pl->len_key;
    p.len_hist = (pl->flags & NB_FLAG_NO_LIST_SORT) ? nullptr : pl->len_hist;
    p.r2cut = r_inner2;
    p.stale_search2 = stale_search2;
    // work_prune and inner_count were reset by the snapshot gather before this launch
    int blocks = pl->num_sms * 4;
    blocks = min(blocks, (pl->nc_max + kPruneThreads / 32 - 1) / (kPruneThreads / 32));
    if (p.vt_slot)
        k_prune<true><<<max(blocks, 1), kPruneThreads, 0, s>>>(p);
    else
        k_prune<false><<<max(blocks, 1), kPruneThreads, 0, s>>>(p);
    return cudaGetLastError();
}
