// Rolling prune (§III-A, "Prune-only kernel"): outer list at rlist ->
// inner list at r_inner, with atom-pair in-range masks. As in the paper's
// post-pruning list sorting, the prune also computes the list-size
// histogram that the sort needs.
//
// One warp per i-cluster (work counter). The outer entries are taken 32 at
// a time, one per lane; the warp first stages the 32 j clusters in shared
// memory (coalesced cp.async, 8 lanes per cluster), then each lane tests
// the 64 atom pairs of its entry with the FP32 distance contract, on the
// packed two-wide FP32 instructions (the 8 rows of ci as 4 row pairs in
// registers, against each j atom). Each lane-wise operation is the IEEE
// operation of the scalar contract, so the decisions are those of
// nb_r2(...) < r2cut. Entries with an empty mask are dropped. The inner
// list of ci is written to its own buffer at the same offset as its outer
// list (the kept entries fill a prefix of that range).
#include "nb_pair_x2.cuh"
#include "nb_warp.cuh"

namespace {

constexpr int kPruneThreads = 128;
constexpr int kPruneWarps = kPruneThreads / 32;
constexpr int kPruneCtasPerSm = 6;  // 80 registers per thread (a few bytes spill; faster than 4 CTAs at 106)

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
    int *nl_list;        // with a halo: the halves (2 ci + h) that have non-local tiles, appended
    int pad_slot;        // a slot that never holds an atom (far away, q = 0)
    int *len_key;        // [nc_max] work of each i-cluster for the force kernel
    int *len_hist;       // [NB_LEN_BINS] histogram of len_key, or NULL (no sorting)
    const unsigned char *clus_home;  // with a halo: bit b = slot b of the cluster holds a home atom
    int reg_stride;      // 2 nc_max: halves per region of half_start / half_len
    float r2cut;
    float stale_search2;
};

// Ring of staged j atoms per warp, half and part: it holds up to 31 atoms
// left from full tiles plus one pass of kSub entries (8 atoms each); a chunk
// whose atoms fit goes in one pass of all 32 entries.
template <int NPART>
struct Ring {
    static constexpr int kSub = NPART == 1 ? 16 : 8;
    static constexpr int kStage = NPART == 1 ? 256 : 128;
    static_assert(kStage >= 31 + 8 * kSub, "ring too small");
};

// Writes ntiles (<= 4) gathered tiles from the 8 ntiles staged atoms at ring
// position head (each a (slot word, mask word) pair): lane l takes atom l, i.e. column p = l & 7 of tile l >> 3.
// Each staged atom keeps its entry's 4 x 8 mask word of the half; its column
// b in that word is the low 3 bits of its slot, so its rows (bits b, 8 + b,
// 16 + b, 24 + b) shifted to column p are its part of the tile's mask, and
// the 8 lanes of a tile OR theirs together.
template <int STAGE>
__device__ __forceinline__ void flush_tiles(const uint2 *ring, int head, int vt, int ntiles, int lane,
                                            const PruneParams &p) {
    const uint2 a = ring[(head + lane) & (STAGE - 1)];  // (slot word, mask word)
    const int v = (int)a.x;
    const int pcol = lane & 7, t = lane >> 3;
    unsigned c = ((a.y >> (a.x & 7u)) & 0x01010101u) << pcol;
    c |= __shfl_xor_sync(0xffffffffu, c, 1);
    c |= __shfl_xor_sync(0xffffffffu, c, 2);
    c |= __shfl_xor_sync(0xffffffffu, c, 4);
    if (t < ntiles) {
        p.vt_slot[8 * (size_t)vt + lane] = v;
        if (pcol == 0) p.vt_mask[vt + t] = c;
    }
}

// The new masks of one entry (the lane's): its 64 atom pairs against r2cut,
// ANDed with the entry's old masks. rx/ry/rz: rows (2k, 2k + 1) of ci as
// packed pairs; xj: the j cluster's 8 atoms (shared memory); S: the entry's
// shift (0 for the center, where adding it is exact).
// r2 < r2cut exactly when fl(r2 - r2cut) is negative: the difference of two
// distinct finite floats rounds to a nonzero value of its sign (subnormals
// are kept), and equal values give +0. So one packed subtraction decides two
// pairs, and a funnel shift moves each sign bit into the row's mask byte; j
// atoms are taken from 7 down to 0 so that atom b ends at bit b. Without
// SHIFT (every entry of the chunk at the center image) the addition of
// S = 0 is left out: it changes no difference but the sign of a zero.
template <bool SHIFT>
__device__ __forceinline__ uint2 test_entry(const int4 e, const float2 (&rx)[4], const float2 (&ry)[4],
                                            const float2 (&rz)[4], const float4 *xj, const float4 S, float r2cut) {
    const float2 Sx = nb_f2(S.x), Sy = nb_f2(S.y), Sz = nb_f2(S.z), nr2cut = nb_f2(-r2cut);
    unsigned ma[4] = {0u, 0u, 0u, 0u}, mb[4] = {0u, 0u, 0u, 0u};  // rows 2k and 2k + 1
#pragma unroll
    for (int b = NB_CLUSTER - 1; b >= 0; --b) {
        const float4 x = xj[b];
        const float2 nx = nb_f2(-x.x), ny = nb_f2(-x.y), nz = nb_f2(-x.z);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 dx = __fadd2_rn(rx[k], nx), dy = __fadd2_rn(ry[k], ny), dz = __fadd2_rn(rz[k], nz);
            if (SHIFT) {
                dx = __fadd2_rn(dx, Sx);
                dy = __fadd2_rn(dy, Sy);
                dz = __fadd2_rn(dz, Sz);
            }
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 t = __fadd2_rn(r2, nr2cut);
            ma[k] = __funnelshift_l(__float_as_uint(t.x), ma[k], 1);
            mb[k] = __funnelshift_l(__float_as_uint(t.y), mb[k], 1);
        }
    }
    // bit a * 8 + b: rows 0-3 in the low word, rows 4-7 in the high word
    const unsigned lo = ma[0] | (mb[0] << 8) | (ma[1] << 16) | (mb[1] << 24);
    const unsigned hi = ma[2] | (mb[2] << 8) | (ma[3] << 16) | (mb[3] << 24);
    return make_uint2(lo & (unsigned)e.z, hi & (unsigned)e.w);
}

// One warp per i-cluster. The outer entries of ci are read 32 at a time
// (one per lane, coalesced); lane t tests entry t and keeps its new masks,
// and the kept entries are written back compacted and coalesced.
// With a halo (NPART = 2) the tiles of each half are gathered in two sets:
// pairs of two home atoms (region 0) and the rest (region 1).
template <bool TILES, int NPART>
__global__ void __launch_bounds__(kPruneThreads, kPruneCtasPerSm) k_prune(PruneParams p) {
    constexpr int kStage = Ring<NPART>::kStage, kSub = Ring<NPART>::kSub, kSets = 2 * NPART;
    // the j clusters of a chunk's entries; one float4 of padding per entry keeps the lanes'
    // 16-byte reads of one atom index free of bank conflicts
    __shared__ float4 s_xj[kPruneWarps][32][NB_CLUSTER + 1];
    __shared__ uint2 s_ring[kPruneWarps][kSets][kStage];  // staged atoms: (slot word, entry's mask word)
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
    const unsigned lanebit = 1u << lane;
    const int nc = p.st->nc;
    const unsigned nwarps = gridDim.x * kPruneWarps;
    for (unsigned it = 0;; ++it) {
        // a warp's first i-cluster is its own index in the grid, later ones come from the counter
        unsigned w = blockIdx.x * kPruneWarps + warp;
        if (it > 0) {
            unsigned a = 0;
            if (lane == 0) a = atomicAdd(&p.st->work_prune, 1u);
            w = __shfl_sync(0xffffffffu, a, 0) + nwarps;
        }
        if (w >= (unsigned)nc) break;
        const int ci = (int)w;
        const float4 *shift = p.sys_shift + 27 * p.clus_sys[ci];
        const int k0 = p.ci_start[ci], n = p.ci_len_outer[ci];
        // tiles of set r (part r >> 1, half r & 1) go to [2 NPART k0 + r n, + n):
        // each entry adds at most 8 atoms to a set
        float2 rx[4], ry[4], rz[4];  // rows (2k, 2k + 1) of ci
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 ra = p.xq[ci * NB_CLUSTER + 2 * k], rb = p.xq[ci * NB_CLUSTER + 2 * k + 1];
            rx[k] = make_float2(ra.x, rb.x);
            ry[k] = make_float2(ra.y, rb.y);
            rz[k] = make_float2(ra.z, rb.z);
        }
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
            int4 e = make_int4(0, NB_SHIFT_CENTER, 0, 0);
            if (lane < cnt) e = p.outer[k0 + base + lane];
            // stage the chunk's j clusters: 8 lanes copy one cluster (128 contiguous bytes)
            __syncwarp();  // the previous chunk's reads of s_xj are done
#pragma unroll
            for (int k = 0; k < 8; ++k) {  // 4 clusters per pass
                const int t = 4 * k + (lane >> 3);
                const int cj = __shfl_sync(0xffffffffu, e.x, t);
                if (t < cnt) cp_async16(&s_xj[warp][t][lane & 7], p.xq + cj * NB_CLUSTER + (lane & 7));
            }
            cp_async_wait_all();
            __syncwarp();
            uint2 mine = make_uint2(0u, 0u);
            if (__any_sync(0xffffffffu, e.y != NB_SHIFT_CENTER)) {
                if (lane < cnt) mine = test_entry<true>(e, rx, ry, rz, s_xj[warp][lane], shift[e.y], p.r2cut);
            } else if (lane < cnt) {
                mine = test_entry<false>(e, rx, ry, rz, s_xj[warp][lane], make_float4(0.f, 0.f, 0.f, 0.f), p.r2cut);
            }
            const bool keep = lane < cnt && (mine.x | mine.y) != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
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
            if (TILES) {
                // In entry order (atoms of one entry stay together, so a tile draws on few
                // clusters): an exclusive scan of the per-entry atom counts places each lane's
                // atoms in its set's ring; once 32 atoms are staged, 4 full tiles leave together.
                // The counts of two sets share one scan (16-bit fields; a set gains at most 256).
                unsigned mhr[kSets], colr[kSets];
                int cr[kSets], inclr[kSets], totr[kSets];
#pragma unroll
                for (int r = 0; r < kSets; ++r) {
                    const int h = r & 1, part = r >> 1;
                    unsigned mh = lane < cnt ? (h ? mine.y : mine.x) : 0u;
                    if (NPART == 2) mh &= part ? ~(h ? loc_hi : loc_lo) : (h ? loc_hi : loc_lo);
                    mhr[r] = mh;
                    colr[r] = (mh | (mh >> 8) | (mh >> 16) | (mh >> 24)) & 0xffu;
                    cr[r] = __popc(colr[r]);
                }
#pragma unroll
                for (int r = 0; r < kSets; r += 2) {
                    int v = cr[r] | (cr[r + 1] << 16);
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += u;
                    }
                    const int t = __shfl_sync(0xffffffffu, v, 31);
                    inclr[r] = v & 0xffff;
                    inclr[r + 1] = v >> 16;
                    totr[r] = t & 0xffff;
                    totr[r + 1] = t >> 16;
                }
                const unsigned sbase = (unsigned)(e.x * NB_CLUSTER) | ((unsigned)e.y << 27);
#pragma unroll
                for (int r = 0; r < kSets; ++r) {
                    if (totr[r] == 0) continue;
                    // one pass over all 32 entries while the ring has room (nearly always: fill
                    // <= 31 and a chunk adds 8 atoms per entry at most, about 4.5 on water);
                    // else kSub entries at a time, flushing in between
                    const int ngroups = fill[r] + totr[r] <= kStage ? 1 : 32 / kSub;
                    const int gsize = 32 / ngroups;
                    for (int sp = 0; sp < ngroups; ++sp) {
                        const int before = sp == 0 ? 0 : __shfl_sync(0xffffffffu, inclr[r], sp * gsize - 1);
                        const int upto = __shfl_sync(0xffffffffu, inclr[r], sp * gsize + gsize - 1);
                        if (lane / gsize == sp) {
                            int k = head[r] + fill[r] + inclr[r] - cr[r] - before;
                            const unsigned col = colr[r];
#pragma unroll
                            for (int bb = 0; bb < 8; ++bb) {
                                if ((col >> bb) & 1u) {
                                    s_ring[warp][r][k & (kStage - 1)] = make_uint2(sbase + (unsigned)bb, mhr[r]);
                                    ++k;
                                }
                            }
                        }
                        fill[r] += upto - before;
                        __syncwarp();
                        while (fill[r] >= 32) {
                            flush_tiles<kStage>(s_ring[warp][r], head[r], 2 * NPART * k0 + r * n + ntile[r], 4,
                                                lane, p);
                            __syncwarp();
                            head[r] += 32;
                            fill[r] -= 32;
                            ntile[r] += 4;
                        }
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
                    s_ring[warp][r][(head[r] + lane) & (kStage - 1)] =
                        make_uint2((unsigned)p.pad_slot | ((unsigned)NB_SHIFT_CENTER << 27), 0u);
                }
                __syncwarp();
                flush_tiles<kStage>(s_ring[warp][r], head[r], 2 * NPART * k0 + r * n + ntile[r], nt, lane, p);
                ntile[r] += nt;
            }
            if (lane == 0) {
                const size_t hidx = (size_t)(r >> 1) * p.reg_stride + 2 * ci + (r & 1);
                p.half_start[hidx] = 2 * NPART * k0 + r * n;
                p.half_len[hidx] = ntile[r];
                // the non-local force launch takes its work from this list, not from every half
                if (NPART == 2 && (r >> 1) == 1 && ntile[r] > 0)
                    p.nl_list[atomicAdd(&p.st->nl_count, 1u)] = 2 * ci + (r & 1);
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
                atomicAdd(&p.st->tile_count, (unsigned long long)key);
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
    p.nl_list = pl->nl_list;
    p.pad_slot = pl->nc_max * NB_CLUSTER;
    p.len_key = pl->len_key;
    p.len_hist = (pl->flags & NB_FLAG_NO_LIST_SORT) ? nullptr : pl->len_hist;
    p.r2cut = r_inner2;
    p.stale_search2 = stale_search2;
    // work_prune and inner_count were reset by the snapshot gather before this launch
    int blocks = pl->num_sms * kPruneCtasPerSm;
    blocks = min(blocks, (pl->nc_max + kPruneWarps - 1) / kPruneWarps);
    p.clus_home = pl->clus_home;
    p.reg_stride = 2 * pl->nc_max;
    if (!p.vt_slot) return nb_launch_pdl(k_prune<false, 1>, max(blocks, 1), kPruneThreads, 0, s, p);
    if (pl->vt_parts == 2) return nb_launch_pdl(k_prune<true, 2>, max(blocks, 1), kPruneThreads, 0, s, p);
    return nb_launch_pdl(k_prune<true, 1>, max(blocks, 1), kPruneThreads, 0, s, p);
}
