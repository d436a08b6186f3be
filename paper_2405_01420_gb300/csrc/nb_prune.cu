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
    int *vt_slot;        // [2 parts * 2 cap * 8] gathered j slots (shift index in the top 5 bits)
    unsigned *vt_mask;   // [2 parts * 2 cap] 4 x 8 in-range bits (bit a*8 + p)
    int *half_start;     // [2 parts][2 nc_max]
    int *half_len;       // [2 parts][2 nc_max]
    int pad_slot;        // a slot that never holds an atom (far away, q = 0)
    int *len_key;        // [nc_max] work of each i-cluster for the force kernel
    int *len_hist;       // [NB_LEN_BINS] histogram of len_key, or NULL (no sorting)
    const unsigned char *clus_home;  // with a halo: bit b = slot b of the cluster holds a home atom
    int reg_stride;      // 2 nc_max: halves per region of half_start / half_len
    float r2cut;
    float stale_search2;
};

// Ring of staged j atoms per warp, half and part: it holds up to 31 atoms
// left from full tiles plus one pass of kSub entries (8 atoms each).
template <int NPART>
struct Ring {
    static constexpr int kSub = NPART == 1 ? 16 : 8;
    static constexpr int kStage = NPART == 1 ? 256 : 128;
    static_assert(kStage >= 31 + 8 * kSub, "ring too small");
};

// Writes ntiles (<= 4) gathered tiles from the 8 ntiles staged atoms at ring
// position head: lane l takes atom l, i.e. column p = l & 7 of tile l >> 3.
// Each staged atom keeps its entry's 4 x 8 mask word of the half; its column
// b in that word is the low 3 bits of its slot, so its rows (bits b, 8 + b,
// 16 + b, 24 + b) shifted to column p are its part of the tile's mask, and
// the 8 lanes of a tile OR theirs together.
template <int STAGE>
__device__ __forceinline__ void flush_tiles(const int *ring_slot, const unsigned *ring_mask, int head, int vt,
                                            int ntiles, int lane, const PruneParams &p) {
    const int idx = (head + lane) & (STAGE - 1);
    const int v = ring_slot[idx];
    const int pcol = lane & 7, t = lane >> 3;
    unsigned c = ((ring_mask[idx] >> ((unsigned)v & 7u)) & 0x01010101u) << pcol;
    c |= __shfl_xor_sync(0xffffffffu, c, 1);
    c |= __shfl_xor_sync(0xffffffffu, c, 2);
    c |= __shfl_xor_sync(0xffffffffu, c, 4);
    if (t < ntiles) {
        p.vt_slot[8 * (size_t)vt + lane] = v;
        if (pcol == 0) p.vt_mask[vt + t] = c;
    }
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
// With a halo (NPART = 2) the tiles of each half are gathered in two sets:
// pairs of two home atoms (region 0) and the rest (region 1).
template <bool TILES, int NPART>
__global__ void __launch_bounds__(kPruneThreads) k_prune(PruneParams p) {
    constexpr int kStage = Ring<NPART>::kStage, kSub = Ring<NPART>::kSub, kSets = 2 * NPART;
    __shared__ int4 s_ent[kPruneThreads / 32][32];
    __shared__ int s_rslot[kPruneThreads / 32][kSets][kStage];
    __shared__ unsigned s_rmask[kPruneThreads / 32][kSets][kStage];
    nb_pdl_wait();  // launched with nb_launch_pdl: the prune's gather has completed from here on
    nb_pdl_release();
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
        // tiles of set r (part r >> 1, half r & 1) go to [2 NPART k0 + r n, + n):
        // each entry adds at most 8 atoms to a set
        const float4 xi1 = p.xq[ci * NB_CLUSTER + a1], xi2 = p.xq[ci * NB_CLUSTER + a2];
        unsigned rows_lo = 0u, rows_hi = 0u;  // home rows of ci as byte masks (rows 0-3 / 4-7)
        if (NPART == 2) {
            const unsigned hci = p.clus_home[ci];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                rows_lo |= ((hci >> a) & 1u) ? 0xffu << (8 * a) : 0u;
                rows_hi |= ((hci >> (a + 4)) & 1u) ? 0xffu << (8 * a) : 0u;
            }
        }
        int out = 0;
        int head[kSets], fill[kSets], ntile[kSets];
#pragma unroll
        for (int r = 0; r < kSets; ++r) head[r] = fill[r] = ntile[r] = 0;
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
            // Gather, per half (and part), the j atoms in range of any of its 4 rows.
            unsigned loc_lo = 0xffffffffu, loc_hi = 0xffffffffu;  // local pairs of the lane's entry
            if (NPART == 2) {
                const unsigned hjw = (lane < cnt ? (unsigned)p.clus_home[e.x] : 0u) * 0x01010101u;
                loc_lo = hjw & rows_lo;
                loc_hi = hjw & rows_hi;
            }
#pragma unroll
            for (int r = 0; r < (TILES ? kSets : 0); ++r) {
                // in entry order (atoms of one entry stay together, so a tile
                // draws on few clusters), kSub entries at a time: an exclusive
                // scan of the per-entry counts places each lane's atoms; once
                // 32 atoms are staged, 4 full tiles leave together
                const int h = r & 1, part = r >> 1;
                unsigned mh = lane < cnt ? (h ? mine.y : mine.x) : 0u;
                if (NPART == 2) mh &= part ? ~(h ? loc_hi : loc_lo) : (h ? loc_hi : loc_lo);
                const unsigned colh = (mh | (mh >> 8) | (mh >> 16) | (mh >> 24)) & 0xffu;
                const unsigned sbase = (unsigned)(e.x * NB_CLUSTER) | ((unsigned)e.y << 27);
#pragma unroll
                for (int sp = 0; sp < 32 / kSub; ++sp) {
                    const unsigned col = lane / kSub == sp ? colh : 0u;
                    const int c = __popc(col);
                    int incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const int total = __shfl_sync(0xffffffffu, incl, 31);
                    if (total == 0) continue;
                    const int pos0 = head[r] + fill[r] + incl - c;
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) {
                        if ((col >> bb) & 1u) {
                            const int idx = (pos0 + __popc(col & ((1u << bb) - 1u))) & (kStage - 1);
                            s_rslot[warp][r][idx] = (int)(sbase + (unsigned)bb);
                            s_rmask[warp][r][idx] = mh;
                        }
                    }
                    fill[r] += total;
                    __syncwarp();
                    while (fill[r] >= 32) {
                        flush_tiles<kStage>(s_rslot[warp][r], s_rmask[warp][r], head[r],
                                            2 * NPART * k0 + r * n + ntile[r], 4, lane, p);
                        __syncwarp();
                        head[r] += 32;
                        fill[r] -= 32;
                        ntile[r] += 4;
                    }
                }
            }
        }
        // the rest of each set: its full tiles and a last one padded with a
        // slot that holds no atom
#pragma unroll
        for (int r = 0; r < (TILES ? kSets : 0); ++r) {
            if (fill[r] > 0) {
                const int nt = (fill[r] + 7) >> 3;
                if (lane >= fill[r] && lane < 8 * nt) {
                    const int idx = (head[r] + lane) & (kStage - 1);
                    s_rslot[warp][r][idx] = (int)((unsigned)p.pad_slot | ((unsigned)NB_SHIFT_CENTER << 27));
                    s_rmask[warp][r][idx] = 0u;
                }
                __syncwarp();
                flush_tiles<kStage>(s_rslot[warp][r], s_rmask[warp][r], head[r], 2 * NPART * k0 + r * n + ntile[r], nt,
                                    lane, p);
                ntile[r] += nt;
            }
            if (lane == 0) {
                const size_t hidx = (size_t)(r >> 1) * p.reg_stride + 2 * ci + (r & 1);
                p.half_start[hidx] = 2 * NPART * k0 + r * n;
                p.half_len[hidx] = ntile[r];
            }
        }
        __syncwarp();
        if (lane == 0) {
            p.ci_len_inner[ci] = out;
            atomicAdd(&p.st->inner_count, (unsigned long long)out);
            // post-prune sorting: the force kernel's work for ci and its histogram
            int key = out;
            if (TILES) {
                key = 0;
#pragma unroll
                for (int r = 0; r < kSets; ++r) key += ntile[r];
            }
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
    p.clus_home = pl->clus_home;
    p.reg_stride = 2 * pl->nc_max;
    if (!p.vt_slot) return nb_launch_pdl(k_prune<false, 1>, max(blocks, 1), kPruneThreads, 0, s, p);
    if (pl->vt_parts == 2) return nb_launch_pdl(k_prune<true, 2>, max(blocks, 1), kPruneThreads, 0, s, p);
    return nb_launch_pdl(k_prune<true, 1>, max(blocks, 1), kPruneThreads, 0, s, p);
}
