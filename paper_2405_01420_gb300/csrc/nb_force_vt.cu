// Force kernel over gathered tiles (the pruned list in its packed form).
//
// After a prune, each half i-cluster (rows 0-3 or 4-7 of an 8-atom cluster)
// has a list of 4 x 8 tiles whose 8 j atoms are gathered from all its
// cluster pairs: only j atoms within r_inner of at least one of the 4 rows
// appear, each with its own periodic shift (nb_prune.cu writes them). The
// arithmetic per pair is that of the cluster-pair kernel (nb_pair with
// d = (y_a - y_b) + S), so both kernels make the same in-range decisions.
//
// Layout (j-stationary): a warp takes one half at a time and reads its
// tiles in groups of 4, i.e. 32 j atoms, one per lane; each lane computes
// its j atom against the half's 4 i rows. On water at rc 1.0 / r_inner
// 1.04 nm about 60% of these pair slots are in range, against 40% for 8 x 8
// cluster tiles with empty half-tiles skipped.
//
//  - The pair arithmetic runs on the packed two-wide FP32 instructions:
//    rows (0, 1) and (2, 3) of the half are two row pairs, each evaluated
//    against the lane's j atom by nb_pair_x2 (one packed operation for two
//    pairs, same rounding per pair as nb_pair). The kernel is bound by
//    instruction issue, and packing halves the issue slots of the FP32 work.
//  - j data (coordinates and charge, type, mask word) of group g + 1 are
//    copied into shared memory with cp.async from the start of group g
//    (their slot words were loaded one group earlier still); the
//    shift vectors come from a per-warp shared copy of the system's 27; the
//    row pairs' positions and charges and their LJ coefficients by j type
//    sit in per-warp shared tables, already in packed order.
//  - j forces stay in registers over the 4 rows and go out with one
//    16-byte vector atomic per lane (fsort is float4 per slot).
//  - i forces stay in registers over the whole half and are reduced across
//    the warp at its end, one vector atomic per row.
//  - Energies: FP32 over a half (per lane, then across the warp), FP64
//    across halves in a per-warp shared pair (no registers held across
//    halves), FP64 atomics per system when the warp moves to another
//    system or finishes.
//  - Every half comes from the work counter, the first too: taking each
//    warp's first half from its grid index instead was 1 us slower at
//    96,000 atoms (the counter spreads the largest halves over the SMs as
//    they free up).
#include "nb_pair_x2.cuh"
#include "nb_warp.cuh"

namespace {

struct VtParams {
    const float4 *xq;
    const int *tsort;
    float *fsort;             // float4 per slot, viewed as floats
    const int *vt_slot;       // 8 per tile: slot | shift << 27
    const unsigned *vt_mask;  // 4 x 8 bits per tile
    const int *half_start;
    const int *half_len;
    const int *order;         // i-clusters by decreasing list length, or NULL
    const float *ljparams;
    nb_dev_state *st;
    double *energies;         // [2 nsys]
    const float4 *sys_shift;  // [27 nsys]
    const int *clus_sys;
    int ntype;
    float rc6inv, rc12inv;
    nb_coul cc;
    nb_coul2 cc2;             // the same constants in packed form
    float stale_prune2;
    int pad_slot;             // never holds an atom: far away, q = 0, type 0
    int reg0, nreg;           // regions of gathered tiles to compute (0 local or all, 1 non-local)
    int reg_stride;           // 2 nc_max: halves per region in half_start / half_len
    const int *nl_list;       // with a halo: the halves with non-local tiles (the prune's list), else NULL
    int finalize;             // move the displacement maxima of this evaluation to last_*
};

// Adds a warp's energies of one system (Coulomb in e[0], LJ in e[1]) to
// that system's pair (E_LJ, E_C) and clears them; lane 0 only.
__device__ __forceinline__ void flush_energies_vt(double *e, double *out) {
    atomicAdd(&out[0], e[1]);
    atomicAdd(&out[1], e[0]);
    e[0] = 0.0;
    e[1] = 0.0;
}

// Per-lane staging of one group of 32 gathered j atoms (4 tiles of 8).
struct VtStage {
    float4 xj[32];
    int tj[32];
    unsigned m[32];
};

// The lane's slot word of group g of the half with tiles [t0, t1): its j
// atom's slot and shift, or the pad slot past the end (the load then reads
// tile t0, so that no lane branches).
__device__ __forceinline__ int slot_word(const VtParams &p, int t0, int t1, int g, int lane) {
    const int tile = t0 + 4 * g + (lane >> 3);
    const bool live = tile < t1;
    const int tc = live ? tile : t0;
    const int w = p.vt_slot[8 * (size_t)tc + (lane & 7)];
    return live ? w : (int)((unsigned)p.pad_slot | ((unsigned)NB_SHIFT_CENTER << 27));
}

// Issues the copies of group g (slot word v) into st: the tile's mask word
// (zero-filled past the end), the j atom's coordinates and charge, its type.
__device__ __forceinline__ void stage_copies(const VtParams &p, VtStage &st, int v, int t0, int t1, int g,
                                             int lane) {
    const int tile = t0 + 4 * g + (lane >> 3);
    const bool live = tile < t1;
    cp_async4_zfill(&st.m[lane], p.vt_mask + (live ? tile : t0), live ? 4u : 0u);
    const int slot = v & 0x07ffffff;
    cp_async16(&st.xj[lane], p.xq + slot);
    cp_async4(&st.tj[lane], p.tsort + slot);
}

// j-stationary kernel over gathered tiles. A warp takes one half i-cluster
// (4 i rows) at a time; its tiles are read in groups of 4 (32 j atoms, one
// per lane), and each lane computes its j atom against the 4 rows, two row
// pairs of packed arithmetic. j forces stay in registers for the 4 pairs
// and go out with one 16-byte vector atomic per lane (fsort is float4 per
// slot); i forces stay in registers for the whole half and are reduced
// across the warp at its end. Group g + 1 is copied (cp.async) into the
// other buffer while group g is computed, and group g + 2's slot words load
// meanwhile.
// Dynamic shared memory: the ntype x ntype LJ table, then per warp 3 float4
// per j type (see s_lj2).
// 640 / THREADS resident CTAs per SM (5 of 128 threads, the default shape)
// leave up to 102 registers per thread (89 used, no spills): the 4 rows'
// forces and the j atom's data stay in registers; the rows' positions,
// charges and LJ coefficients are read from the per-warp shared tables.
// 6 CTAs at 80 registers (and 3 of 256) were 3.5-4 us slower at 96,000
// atoms, 4 CTAs at up to 128 registers 0.5 us slower.
template <bool ENERGY, bool COUNT, int THREADS, int COUL>
__global__ void __launch_bounds__(THREADS, 640 / THREADS) k_force_vt(VtParams p) {
    constexpr int kWarps = THREADS / 32;
    extern __shared__ float4 s_lj[];
    __shared__ VtStage s_st[kWarps][2];
    __shared__ float4 s_shift[kWarps][27];  // the warp's copy of its system's shift vectors
    int shift_sys = -1;
    __shared__ float4 s_xi[kWarps][4];
    __shared__ int s_tr[kWarps][4];
    __shared__ float4 s_xp[kWarps][2][2];  // row pair k: (x_a, x_b, y_a, y_b), (z_a, z_b, fq_a, fq_b)
    __shared__ double s_e[kWarps][2];      // the warp's energies of its current system: Coulomb, LJ
    nb_pdl_wait();  // launched with nb_launch_pdl: the gather has completed from here on
    nb_pdl_release();
    const int nt2 = p.ntype * p.ntype;
    for (int k = threadIdx.x; k < nt2; k += blockDim.x) {
        const float c6 = p.ljparams[2 * k], c12 = p.ljparams[2 * k + 1];
        s_lj[k] = make_float4(c6, c12, c12 * p.rc12inv - c6 * p.rc6inv, 0.0f);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned ds = p.st->cur_d2_search, dp = p.st->cur_d2_prune;
        if (p.finalize) {
            p.st->last_d2_search = ds;
            p.st->last_d2_prune = dp;
            p.st->cur_d2_search = 0u;
            p.st->cur_d2_prune = 0u;
        }
        if (__uint_as_float(dp) > p.stale_prune2) atomicOr(&p.st->err, NB_DEV_STALE_PRUNE);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per warp, for the current half, by j type t: (C6, C6, C12, C12) of
    // row pairs (0, 1) and (2, 3) at [3t], [3t + 1], minus the 4 rows' LJ
    // shifts at [3t + 2]
    float4 *s_lj2 = s_lj + nt2 + 3 * p.ntype * warp;
    // Work items: region 0 (every pair without a halo, the local pairs with one) is every half, in
    // the list order; region 1 (non-local) is the prune's list of the halves that have such tiles
    const unsigned nhalf = 2u * (unsigned)p.st->nc;  // halves per region
    const unsigned n0 = p.reg0 == 0 ? nhalf : 0u;
    const unsigned n1 = p.reg0 + p.nreg == 2 ? (p.nl_list ? p.st->nl_count : nhalf) : 0u;
    const unsigned nwork = n0 + n1;
    if (ENERGY && lane == 0) s_e[warp][0] = s_e[warp][1] = 0.0;
    int cur_sys = -1;
    unsigned cnt = 0;

    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&p.st->work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        unsigned reg = 0u, hw = 0u;
        int ci = 0;
        if (w < n0) {
            hw = w;
            ci = p.order ? p.order[hw >> 1] : (int)(hw >> 1);
        } else if (w < nwork) {
            reg = 1u;
            hw = p.nl_list ? (unsigned)p.nl_list[w - n0] : w - n0;
            ci = (int)(hw >> 1);
        }
        const int h = (int)(hw & 1u);
        const int csys = (w < nwork) ? p.clus_sys[ci] : -1;
        if (ENERGY && csys != cur_sys) {
            if (cur_sys >= 0 && lane == 0) flush_energies_vt(s_e[warp], p.energies + 2 * cur_sys);
            cur_sys = csys;
        }
        if (w >= nwork) break;
        const size_t hidx = (size_t)reg * p.reg_stride + 2 * ci + h;
        const int t0 = p.half_start[hidx], t1 = t0 + p.half_len[hidx];
        if (t1 <= t0) continue;
        if (csys != shift_sys) {
            if (lane < 27) s_shift[warp][lane] = p.sys_shift[27 * csys + lane];
            shift_sys = csys;
        }
        const int ibase = ci * NB_CLUSTER + 4 * h;
        int v = slot_word(p, t0, t1, 0, lane);
        stage_copies(p, s_st[warp][0], v, t0, t1, 0, lane);
        int vnext = slot_word(p, t0, t1, 1, lane);
        if (lane < 4) {
            const float4 x = p.xq[ibase + lane];
            s_xi[warp][lane] = make_float4(x.x, x.y, x.z, x.w * NB_COULOMB_F);
            s_tr[warp][lane] = p.tsort[ibase + lane] * p.ntype;
        }
        float2 fix[2], fiy[2], fiz[2];  // row pair k: rows 2k (.x) and 2k + 1 (.y)
#pragma unroll
        for (int k = 0; k < 2; ++k) fix[k] = fiy[k] = fiz[k] = make_float2(0.f, 0.f);
        float2 ec2 = make_float2(0.f, 0.f), elj2 = make_float2(0.f, 0.f);
        const int ngroups = (t1 - t0 + 3) >> 2;
        cp_async_wait_all();
        __syncwarp();
        if (lane < 2) {
            const float4 a = s_xi[warp][2 * lane], b = s_xi[warp][2 * lane + 1];
            s_xp[warp][lane][0] = make_float4(a.x, b.x, a.y, b.y);
            s_xp[warp][lane][1] = make_float4(a.z, b.z, a.w, b.w);
        }
        for (int t = lane; t < p.ntype; t += 32) {
            const float4 c0 = s_lj[s_tr[warp][0] + t], c1 = s_lj[s_tr[warp][1] + t];
            const float4 c2 = s_lj[s_tr[warp][2] + t], c3 = s_lj[s_tr[warp][3] + t];
            s_lj2[3 * t + 0] = make_float4(c0.x, c1.x, c0.y, c1.y);
            s_lj2[3 * t + 1] = make_float4(c2.x, c3.x, c2.y, c3.y);
            s_lj2[3 * t + 2] = make_float4(-c0.z, -c1.z, -c2.z, -c3.z);
        }
        __syncwarp();
        for (int g = 0; g < ngroups; ++g) {
            VtStage &cs = s_st[warp][g & 1];
            const float4 xj = cs.xj[lane];
            const float4 S = s_shift[warp][(unsigned)v >> 27];
            const int tj = cs.tj[lane];
            const unsigned mrow = cs.m[lane] >> (lane & 7);  // bit 8a: row a
            const int slot = v & 0x07ffffff;
            const float2 nxjx = nb_f2(-xj.x), nxjy = nb_f2(-xj.y), nxjz = nb_f2(-xj.z), qj = nb_f2(xj.w);
            const float2 Sx = nb_f2(S.x), Sy = nb_f2(S.y), Sz = nb_f2(S.z);
            const float4 nsh = s_lj2[3 * tj + 2];
            float2 gjx = make_float2(0.f, 0.f), gjy = gjx, gjz = gjx;
            // the next group's copies overlap this whole group, and the slot word after it is
            // loaded a group ahead (past the last group: pad copies)
            stage_copies(p, s_st[warp][(g + 1) & 1], vnext, t0, t1, g + 1, lane);
            const int vafter = slot_word(p, t0, t1, g + 2, lane);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float4 xa = s_xp[warp][k][0], xb = s_xp[warp][k][1];
                const int c2 = nb_pair_x2<ENERGY, COUL>(
                    make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xb.x, xb.y),
                    make_float2(xb.z, xb.w), nxjx, nxjy, nxjz, qj, Sx, Sy, Sz, s_lj2[3 * tj + k],
                    k == 0 ? make_float2(nsh.x, nsh.y) : make_float2(nsh.z, nsh.w), ((mrow >> (16 * k)) & 1u) != 0u,
                    ((mrow >> (16 * k + 8)) & 1u) != 0u, p.cc.rc2, p.cc2, fix[k], fiy[k], fiz[k], gjx, gjy, gjz, ec2,
                    elj2);
                if (COUNT) cnt += c2;
            }
            if (slot != p.pad_slot)  // all padding lanes share one slot: no atomics there
                atomicAdd(reinterpret_cast<float4 *>(p.fsort) + slot,
                          make_float4(-(gjx.x + gjx.y), -(gjy.x + gjy.y), -(gjz.x + gjz.y), 0.0f));
            v = vnext;
            vnext = vafter;
            cp_async_wait_all();
            __syncwarp();
        }
        // i forces: row a component c is value 4a + c; lanes 2k hold value k
        float r[16];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            r[8 * k + 0] = fix[k].x;
            r[8 * k + 1] = fiy[k].x;
            r[8 * k + 2] = fiz[k].x;
            r[8 * k + 3] = 0.0f;
            r[8 * k + 4] = fix[k].y;
            r[8 * k + 5] = fiy[k].y;
            r[8 * k + 6] = fiz[k].y;
            r[8 * k + 7] = 0.0f;
        }
        reduce_scatter<16>(r, lane);
        // lane 8a holds row a's x; its y and z sit 2 and 4 lanes up
        const float ry = __shfl_down_sync(0xffffffffu, r[0], 2);
        const float rz = __shfl_down_sync(0xffffffffu, r[0], 4);
        if ((lane & 7) == 0)
            atomicAdd(reinterpret_cast<float4 *>(p.fsort) + ibase + (lane >> 3), make_float4(r[0], ry, rz, 0.0f));
        if (ENERGY) {
            float ec = ec2.x + ec2.y, el = elj2.x + elj2.y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ec += __shfl_xor_sync(0xffffffffu, ec, o);
                el += __shfl_xor_sync(0xffffffffu, el, o);
            }
            if (lane == 0) {
                s_e[warp][0] += (double)ec;
                s_e[warp][1] += (double)el;
            }
        }
        __syncwarp();
    }
    if (COUNT) {
        unsigned long long c64 = cnt;
        for (int o = 16; o > 0; o >>= 1) c64 += __shfl_xor_sync(0xffffffffu, c64, o);
        if (lane == 0) atomicAdd(&p.st->npairs, c64);
    }
}

using VtFn = void (*)(VtParams);
template <bool E, bool C, int K>
VtFn pick_vt_shape(int threads) {
    return threads == 128 ? k_force_vt<E, C, 128, K> : k_force_vt<E, C, 256, K>;
}

template <bool E, bool C>
VtFn pick_vt(int threads, int coul) {
    if (coul == NB_COULK_RF) return pick_vt_shape<E, C, NB_COULK_RF>(threads);
    if (coul == NB_COULK_EWALD_SHIFT) return pick_vt_shape<E, C, NB_COULK_EWALD_SHIFT>(threads);
    return pick_vt_shape<E, C, NB_COULK_EWALD>(threads);
}

struct Occ {
    size_t smem;
    int per_sm;
};
Occ g_vt_occ[3][2][2][2] = {};

}  // namespace

cudaError_t nb_launch_force_vt(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                               double *energies, float stale_prune2, int part, cudaStream_t s) {
    VtParams p;
    // regions: without a halo one (every pair); with one, 0 = local, 1 = non-local
    p.reg0 = part == NB_PART_NONLOCAL ? 1 : 0;
    p.nreg = (part == NB_PART_ALL && pl->vt_parts == 2) ? 2 : 1;
    p.reg_stride = 2 * pl->nc_max;
    p.nl_list = pl->vt_parts == 2 ? pl->nl_list : nullptr;
    p.finalize = part != NB_PART_LOCAL;
    p.xq = pl->xq;
    p.tsort = pl->tsort;
    p.fsort = reinterpret_cast<float *>(pl->fsort);
    p.vt_slot = pl->vt_slot;
    p.vt_mask = pl->vt_mask;
    p.half_start = pl->half_start;
    p.half_len = pl->half_len;
    p.order = pl->sorted ? pl->ci_order : nullptr;
    p.ljparams = ljparams;
    p.st = pl->st;
    p.energies = energies;
    p.sys_shift = pl->sys_shift;
    p.clus_sys = pl->clus_sys;
    p.ntype = ntype;
    const double rc6 = 1.0 / ((double)rc * rc * rc * rc * rc * rc);
    p.rc6inv = (float)rc6;
    p.rc12inv = (float)(rc6 * rc6);
    const int coul = nb_fill_coul(p.cc, rc, beta, pl->coul_kind, pl->eps_rf, pl->coul_flags);
    p.cc2 = nb_pack_coul(p.cc);
    p.stale_prune2 = stale_prune2;
    p.pad_slot = pl->nc_max * NB_CLUSTER;
    const int e = energies ? 1 : 0;
    const int c = (pl->flags & NB_FLAG_COUNT_PAIRS) ? 1 : 0;
    const int threads = pl->force_threads == 256 ? 256 : 128;
    VtFn fn = e ? (c ? pick_vt<true, true>(threads, coul) : pick_vt<true, false>(threads, coul))
                : (c ? pick_vt<false, true>(threads, coul) : pick_vt<false, false>(threads, coul));
    const size_t smem = sizeof(float4) * ((size_t)ntype * ntype + 3 * (size_t)ntype * (threads / 32));
    Occ &occ = g_vt_occ[coul][e][c][threads == 128];
    if (occ.per_sm == 0 || occ.smem != smem) {  // resident CTAs for this LJ table size
        int n = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void *)fn, threads, smem);
        if (err != cudaSuccess) return err;
        occ.smem = smem;
        occ.per_sm = n < 1 ? 1 : n;
    }
    const int per_sm = occ.per_sm;
    const int use = pl->force_blocks_per_sm > 0 ? min(pl->force_blocks_per_sm, per_sm) : per_sm;
    int blocks = pl->num_sms * use;
    blocks = min(blocks, (2 * p.nreg * pl->nc_max + threads / 32 - 1) / (threads / 32));
    return nb_launch_pdl(fn, max(blocks, 1), threads, smem, s, p);
}
