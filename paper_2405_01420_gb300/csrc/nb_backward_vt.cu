// Adjoint over gathered tiles (after a prune): the j-stationary layout of
// the gathered-tile force kernel applied to nb_pair_adj.
//
// A warp takes one half i-cluster (4 i rows) at a time and reads its
// gathered tiles in groups of 32 j atoms, one per lane; each lane computes
// the adjoint of its j atom against the 4 rows.
//  - j side (dL/dx, dL/dq): registers over the 4 rows, then one 16-byte
//    vector atomic per lane into bsort (float4 per slot).
//  - i side: registers over the whole half, reduced across the warp at its
//    end (reduce-scatter), one vector atomic per row.
//  - dL/dC6, dL/dC12: per-lane FP32 accumulators for each (row, j type),
//    kept in shared memory (one column per lane, so a lane's adds never
//    meet another lane's bank), reduced across the warp once per half by a
//    skewed read (lane k sums row k, starting at bank k) and added in FP64
//    to the unsymmetrised [ntype][ntype][2] accumulator. In registers they
//    took 32 of them and held the kernel at 4 warps per scheduler.
// Group g + 1's j data (coordinates and charge, g, type, mask word) are
// copied into shared memory with cp.async from the start of group g, their
// slot words loaded one group earlier still.
#include "nb_pair_x2.cuh"
#include "nb_warp.cuh"

namespace {

constexpr int kBvtThreads = 128;
constexpr int kBvtWarps = kBvtThreads / 32;
constexpr int kBvtCtasPerSm = 4;  // up to 128 registers (115 used); 5 CTAs at 102 were 1.3 us slower at 24k atoms, 6 at 80 slower still

struct BvtParams {
    const float4 *xq;
    const int *tsort;
    const float4 *gsort;
    float4 *bsort;            // (dL/dx, dL/dq) per slot
    double *glj_acc;          // [ntype][ntype][2], unsymmetrised
    const int *vt_slot;       // 8 per tile: slot | shift << 27
    const unsigned *vt_mask;  // 4 x 8 bits per tile
    const int *half_start;
    const int *half_len;
    const int *order;         // i-clusters by decreasing work, or NULL
    const float *ljparams;
    nb_dev_state *st;
    const float4 *sys_shift;  // [27 nsys]
    const int *clus_sys;
    int ntype;
    nb_coul cc;
    nb_coul2 cc2;  // the same constants in packed form
    float k2;  // 2 (2 beta/sqrt(pi)) beta^2
    float stale_prune2;
    int pad_slot;  // never holds an atom: far away, q = 0, type 0
    int nreg;      // regions of gathered tiles (2 with a halo: local, non-local)
    int reg_stride;  // 2 nc_max
};

struct BvtStage {
    float4 xj[32];
    float4 gj[32];
    int tj[32];
    unsigned m[32];
};

// The lane's slot word of group g of the half with tiles [t0, t1): its j
// atom's slot and shift, or the pad slot past the end (the load then reads
// tile t0, so that no lane branches).
__device__ __forceinline__ int slot_word_adj(const BvtParams &p, int t0, int t1, int g, int lane) {
    const int tile = t0 + 4 * g + (lane >> 3);
    const bool live = tile < t1;
    const int tc = live ? tile : t0;
    const int w = p.vt_slot[8 * (size_t)tc + (lane & 7)];
    return live ? w : (int)((unsigned)p.pad_slot | ((unsigned)NB_SHIFT_CENTER << 27));
}

// Issues the copies of group g (slot word v) into st: the tile's mask word
// (zero-filled past the end), the j atom's coordinates and charge, g, type.
__device__ __forceinline__ void stage_adj(const BvtParams &p, BvtStage &st, int v, int t0, int t1, int g, int lane) {
    const int tile = t0 + 4 * g + (lane >> 3);
    const bool live = tile < t1;
    cp_async4_zfill(&st.m[lane], p.vt_mask + (live ? tile : t0), live ? 4u : 0u);
    const int slot = v & 0x07ffffff;
    cp_async16(&st.xj[lane], p.xq + slot);
    cp_async16(&st.gj[lane], p.gsort + slot);
    cp_async4(&st.tj[lane], p.tsort + slot);
}

template <int NT, int COUL>
__global__ void __launch_bounds__(kBvtThreads, kBvtCtasPerSm) k_backward_vt(BvtParams p) {
    constexpr int kAcc = 4 * NT * 2;  // (row a, j type t, C6 / C12) accumulators per lane
    // dynamic: the ntype x ntype LJ table (C6, C12, 0, 0), then per warp, by j type t, the half's
    // row pairs' (C6_a, C6_b, C12_a, C12_b) at [2t + k]
    extern __shared__ float4 s_lj[];
    __shared__ BvtStage s_st[kBvtWarps][2];
    __shared__ float s_acc[kBvtWarps][kAcc][32];  // [value][lane]
    __shared__ float4 s_shift[kBvtWarps][27];
    __shared__ float4 s_xi[kBvtWarps][4];  // (x, y, z, f q)
    __shared__ float4 s_gi[kBvtWarps][4];
    __shared__ int s_tr[kBvtWarps][4];     // LJ table row of each i row
    __shared__ float4 s_xp[kBvtWarps][2][2];  // row pair k: (x_a, x_b, y_a, y_b), (z_a, z_b, fq_a, fq_b)
    __shared__ float4 s_gp[kBvtWarps][2][2];  // row pair k: (gx_a, gx_b, gy_a, gy_b), (gz_a, gz_b, 0, 0)
    nb_pdl_wait();
    nb_pdl_release();
    const int nt2 = p.ntype * p.ntype;
    for (int k = threadIdx.x; k < nt2; k += blockDim.x)
        s_lj[k] = make_float4(p.ljparams[2 * k], p.ljparams[2 * k + 1], 0.0f, 0.0f);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned ds = p.st->cur_d2_search, dp = p.st->cur_d2_prune;
        p.st->last_d2_search = ds;
        p.st->last_d2_prune = dp;
        p.st->cur_d2_search = 0u;
        p.st->cur_d2_prune = 0u;
        if (__uint_as_float(dp) > p.stale_prune2) atomicOr(&p.st->err, NB_DEV_STALE_PRUNE);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nhalf = 2u * (unsigned)p.st->nc;
    const unsigned nwork = nhalf * (unsigned)p.nreg;
    int shift_sys = -1;
    float(*acc)[32] = s_acc[warp];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k][lane] = 0.0f;

    const unsigned nwarps = gridDim.x * kBvtWarps;
    for (unsigned it = 0;; ++it) {
        // a warp's first work item is its own index in the grid, later ones come from the counter
        unsigned w = blockIdx.x * kBvtWarps + warp;
        if (it > 0) {
            unsigned a = 0;
            if (lane == 0) a = atomicAdd(&p.st->work, 1u);
            w = __shfl_sync(0xffffffffu, a, 0) + nwarps;
        }
        if (w >= nwork) break;
        const unsigned reg = w / nhalf, hw = w - reg * nhalf;
        const int ci = p.order ? p.order[hw >> 1] : (int)(hw >> 1);
        const int h = (int)(hw & 1u);
        const size_t hidx = (size_t)reg * p.reg_stride + 2 * ci + h;
        const int t0 = p.half_start[hidx], t1 = t0 + p.half_len[hidx];
        if (t1 <= t0) continue;
        const int csys = p.clus_sys[ci];
        if (csys != shift_sys) {
            if (lane < 27) s_shift[warp][lane] = p.sys_shift[27 * csys + lane];
            shift_sys = csys;
        }
        const int ibase = ci * NB_CLUSTER + 4 * h;
        int v = slot_word_adj(p, t0, t1, 0, lane);
        stage_adj(p, s_st[warp][0], v, t0, t1, 0, lane);
        int vnext = slot_word_adj(p, t0, t1, 1, lane);
        if (lane < 4) {
            const float4 x = p.xq[ibase + lane];
            s_xi[warp][lane] = make_float4(x.x, x.y, x.z, x.w * NB_COULOMB_F);
            s_gi[warp][lane] = p.gsort[ibase + lane];
            s_tr[warp][lane] = p.tsort[ibase + lane] * p.ntype;
        }
        // rows (2k, 2k + 1) of the half in .x, .y of row pair k
        float2 bix[2], biy[2], biz[2], biq[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) bix[k] = biy[k] = biz[k] = biq[k] = make_float2(0.f, 0.f);
        const int ngroups = (t1 - t0 + 3) >> 2;
        cp_async_wait_all();
        __syncwarp();
        if (lane < 2) {
            const float4 a = s_xi[warp][2 * lane], b = s_xi[warp][2 * lane + 1];
            s_xp[warp][lane][0] = make_float4(a.x, b.x, a.y, b.y);
            s_xp[warp][lane][1] = make_float4(a.z, b.z, a.w, b.w);
            const float4 ga = s_gi[warp][2 * lane], gb = s_gi[warp][2 * lane + 1];
            s_gp[warp][lane][0] = make_float4(ga.x, gb.x, ga.y, gb.y);
            s_gp[warp][lane][1] = make_float4(ga.z, gb.z, 0.0f, 0.0f);
        }
        float4 *s_ljp = s_lj + nt2 + 2 * p.ntype * warp;
        for (int t = lane; t < p.ntype; t += 32) {
            const float4 c0 = s_lj[s_tr[warp][0] + t], c1 = s_lj[s_tr[warp][1] + t];
            const float4 c2 = s_lj[s_tr[warp][2] + t], c3 = s_lj[s_tr[warp][3] + t];
            s_ljp[2 * t + 0] = make_float4(c0.x, c1.x, c0.y, c1.y);
            s_ljp[2 * t + 1] = make_float4(c2.x, c3.x, c2.y, c3.y);
        }
        __syncwarp();
        const float2 nk2 = nb_f2(-p.k2);
        for (int g = 0; g < ngroups; ++g) {
            const BvtStage &cs = s_st[warp][g & 1];
            const float4 xj = cs.xj[lane];
            const float4 gj = cs.gj[lane];
            const int tj = cs.tj[lane];
            const unsigned mrow = cs.m[lane] >> (lane & 7);  // bit 8a: row a
            const float4 S = s_shift[warp][(unsigned)v >> 27];
            const int slot = v & 0x07ffffff;
            const float2 nxjx = nb_f2(-xj.x), nxjy = nb_f2(-xj.y), nxjz = nb_f2(-xj.z);
            const float2 ngjx = nb_f2(-gj.x), ngjy = nb_f2(-gj.y), ngjz = nb_f2(-gj.z);
            const float2 qj = nb_f2(xj.w), qj_f = nb_f2(xj.w * NB_COULOMB_F);
            const float2 Sx = nb_f2(S.x), Sy = nb_f2(S.y), Sz = nb_f2(S.z);
            float2 vjx = make_float2(0.f, 0.f), vjy = vjx, vjz = vjx, bjq = vjx;
            // the next group's copies overlap this whole group, and the slot word after it is
            // loaded a group ahead (past the last group: pad copies)
            stage_adj(p, s_st[warp][(g + 1) & 1], vnext, t0, t1, g + 1, lane);
            const int vafter = slot_word_adj(p, t0, t1, g + 2, lane);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float4 xa = s_xp[warp][k][0], xb = s_xp[warp][k][1];
                const float4 ga = s_gp[warp][k][0], gb = s_gp[warp][k][1];
                const float4 lj = s_ljp[2 * tj + k];
                float2 d6, d12;
                nb_pair_adj_x2<COUL>(make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xb.x, xb.y),
                                     make_float2(xb.z, xb.w), make_float2(ga.x, ga.y), make_float2(ga.z, ga.w),
                                     make_float2(gb.x, gb.y), nxjx, nxjy, nxjz, qj, qj_f, ngjx, ngjy, ngjz, Sx, Sy, Sz,
                                     make_float2(lj.x, lj.y), make_float2(lj.z, lj.w),
                                     ((mrow >> (16 * k)) & 1u) != 0u, ((mrow >> (16 * k + 8)) & 1u) != 0u, p.cc.rc2,
                                     p.cc2, nk2, bix[k], biy[k], biz[k], biq[k], vjx, vjy, vjz, bjq, d6, d12);
                // the lane's own columns: tj < ntype <= NT (the gather keeps types in range)
                acc[((2 * k) * NT + tj) * 2 + 0][lane] += d6.x;
                acc[((2 * k) * NT + tj) * 2 + 1][lane] += d12.x;
                acc[((2 * k + 1) * NT + tj) * 2 + 0][lane] += d6.y;
                acc[((2 * k + 1) * NT + tj) * 2 + 1][lane] += d12.y;
            }
            if (slot != p.pad_slot)  // all padding lanes share one slot: no atomics there
                atomicAdd(p.bsort + slot, make_float4(-(vjx.x + vjx.y), -(vjy.x + vjy.y), -(vjz.x + vjz.y),
                                                      bjq.x + bjq.y));
            v = vnext;
            vnext = vafter;
            cp_async_wait_all();
            __syncwarp();
        }
        // i side: value 4a + c (c = x, y, z, q); lane 8a then holds row a's x
        // and finds y, z, q 2, 4 and 6 lanes up
        {
            float r[16];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                r[8 * k + 0] = bix[k].x;
                r[8 * k + 1] = biy[k].x;
                r[8 * k + 2] = biz[k].x;
                r[8 * k + 3] = biq[k].x;
                r[8 * k + 4] = bix[k].y;
                r[8 * k + 5] = biy[k].y;
                r[8 * k + 6] = biz[k].y;
                r[8 * k + 7] = biq[k].y;
            }
            reduce_scatter<16>(r, lane);
            const float ry = __shfl_down_sync(0xffffffffu, r[0], 2);
            const float rz = __shfl_down_sync(0xffffffffu, r[0], 4);
            const float rq = __shfl_down_sync(0xffffffffu, r[0], 6);
            if ((lane & 7) == 0) atomicAdd(p.bsort + ibase + (lane >> 3), make_float4(r[0], ry, rz, rq));
        }
        // LJ gradients: value k = (a NT + t) 2 + c, summed over the 32 lane columns by lane k,
        // which starts at column k so that the 32 lanes read 32 different banks; each value is
        // cleared as it is read
        __syncwarp();
        if (lane < kAcc) {
            float sum = 0.0f;
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                const int col = (i + lane) & 31;
                sum += acc[lane][col];
                acc[lane][col] = 0.0f;
            }
            const int a = lane / (2 * NT), t = (lane >> 1) % NT, c = lane & 1;
            if (t < p.ntype && sum != 0.0f) atomicAdd(&p.glj_acc[2 * (s_tr[warp][a] + t) + c], (double)sum);
        }
        __syncwarp();
    }
}

template <int NT, int COUL>
cudaError_t launch_bvt(nb_pairlist *pl, BvtParams p, cudaStream_t s) {
    const size_t smem = sizeof(float4) * ((size_t)p.ntype * p.ntype + 2 * (size_t)p.ntype * kBvtWarps);
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward_vt<NT, COUL>, kBvtThreads,
                                                                      sizeof(float4) * (16 + 8 * kBvtWarps));
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const int blocks = min(pl->num_sms * per_sm, (2 * p.nreg * pl->nc_max + kBvtWarps - 1) / kBvtWarps);
    return nb_launch_pdl(k_backward_vt<NT, COUL>, max(blocks, 1), kBvtThreads, smem, s, p);
}

}  // namespace

cudaError_t nb_launch_backward_vt(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                                  float stale_prune2, cudaStream_t s) {
    BvtParams p;
    p.xq = pl->xq;
    p.tsort = pl->tsort;
    p.gsort = pl->gsort;
    p.bsort = pl->bsort;
    p.glj_acc = pl->glj_acc;
    p.vt_slot = pl->vt_slot;
    p.vt_mask = pl->vt_mask;
    p.half_start = pl->half_start;
    p.half_len = pl->half_len;
    p.order = pl->sorted ? pl->ci_order : nullptr;
    p.ljparams = ljparams;
    p.st = pl->st;
    p.sys_shift = pl->sys_shift;
    p.clus_sys = pl->clus_sys;
    p.ntype = ntype;
    const int coul = nb_fill_coul(p.cc, rc, beta, pl->coul_kind, pl->eps_rf, pl->coul_flags);
    p.cc2 = nb_pack_coul(p.cc);
    p.k2 = (float)(2.0 * (2.0 * beta / 1.7724538509055159) * (double)beta * beta);
    p.stale_prune2 = stale_prune2;
    p.pad_slot = pl->nc_max * NB_CLUSTER;
    p.nreg = pl->vt_parts == 2 ? 2 : 1;
    p.reg_stride = 2 * pl->nc_max;
    if (coul == NB_COULK_RF) {  // the Ewald shift does not change forces
        if (ntype == 1) return launch_bvt<1, NB_COULK_RF>(pl, p, s);
        if (ntype == 2) return launch_bvt<2, NB_COULK_RF>(pl, p, s);
        return launch_bvt<4, NB_COULK_RF>(pl, p, s);
    }
    if (ntype == 1) return launch_bvt<1, NB_COULK_EWALD>(pl, p, s);
    if (ntype == 2) return launch_bvt<2, NB_COULK_EWALD>(pl, p, s);
    return launch_bvt<4, NB_COULK_EWALD>(pl, p, s);
}
