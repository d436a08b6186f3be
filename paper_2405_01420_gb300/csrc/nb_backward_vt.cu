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
// copied into shared memory with cp.async while group g computes.
#include "nb_pair.cuh"
#include "nb_warp.cuh"

namespace {

constexpr int kBvtThreads = 128;
constexpr int kBvtWarps = kBvtThreads / 32;
constexpr int kBvtCtasPerSm = 5;  // 102 registers per thread

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
    float k2;  // 2 (2 beta/sqrt(pi)) beta^2
    float stale_prune2;
    int pad_slot;  // never holds an atom: far away, q = 0, type 0
    int nreg;      // regions of gathered tiles (2 with a halo: local, non-local)
    int reg_stride;  // 2 nc_max
    int nseg;      // work items per half: its groups of tiles split into nseg ranges
};

struct BvtStage {
    float4 xj[32];
    float4 gj[32];
    int tj[32];
    unsigned m[32];
};

// Issues the copies of the lane's j atom in group g of the half with tiles
// [t0, t1) (t0 < t1); returns its slot word. Past the end: the pad slot and
// a zero-filled mask, with the loads reading tile t0 so that no lane branches.
__device__ __forceinline__ int stage_adj(const BvtParams &p, BvtStage &st, int t0, int t1, int g, int lane) {
    const int tile = t0 + 4 * g + (lane >> 3);
    const bool live = tile < t1;
    const int tc = live ? tile : t0;
    const int w = p.vt_slot[8 * (size_t)tc + (lane & 7)];
    const int v = live ? w : (int)((unsigned)p.pad_slot | ((unsigned)NB_SHIFT_CENTER << 27));
    cp_async4_zfill(&st.m[lane], p.vt_mask + tc, live ? 4u : 0u);
    const int slot = v & 0x07ffffff;
    cp_async16(&st.xj[lane], p.xq + slot);
    cp_async16(&st.gj[lane], p.gsort + slot);
    cp_async4(&st.tj[lane], p.tsort + slot);
    return v;
}

template <int NT, int COUL>
__global__ void __launch_bounds__(kBvtThreads, kBvtCtasPerSm) k_backward_vt(BvtParams p) {
    constexpr int kAcc = 4 * NT * 2;  // (row a, j type t, C6 / C12) accumulators per lane
    extern __shared__ float4 s_lj[];  // (C6, C12, 0, 0)
    __shared__ BvtStage s_st[kBvtWarps][2];
    __shared__ float s_acc[kBvtWarps][kAcc][32];  // [value][lane]
    __shared__ float4 s_shift[kBvtWarps][27];
    __shared__ float4 s_xi[kBvtWarps][4];  // (x, y, z, f q)
    __shared__ float4 s_gi[kBvtWarps][4];
    __shared__ int s_tr[kBvtWarps][4];     // LJ table row of each i row
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
    const unsigned nwork = nhalf * (unsigned)p.nreg * (unsigned)p.nseg;
    int shift_sys = -1;
    float(*acc)[32] = s_acc[warp];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k][lane] = 0.0f;

    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&p.st->work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= nwork) break;
        // work item w: range seg of the groups of half hw of region reg
        const unsigned unit = w / (unsigned)p.nseg, seg = w - unit * (unsigned)p.nseg;
        const unsigned reg = unit / nhalf, hw = unit - reg * nhalf;
        const int ci = p.order ? p.order[hw >> 1] : (int)(hw >> 1);
        const int h = (int)(hw & 1u);
        const size_t hidx = (size_t)reg * p.reg_stride + 2 * ci + h;
        const int th = p.half_start[hidx], nth = p.half_len[hidx];
        const int gh = (nth + 3) >> 2;  // groups of the half
        const int t0 = th + 4 * (int)(((long long)gh * seg) / p.nseg);
        const int t1 = min(th + nth, th + 4 * (int)(((long long)gh * (seg + 1)) / p.nseg));
        if (t1 <= t0) continue;
        const int csys = p.clus_sys[ci];
        if (csys != shift_sys) {
            if (lane < 27) s_shift[warp][lane] = p.sys_shift[27 * csys + lane];
            shift_sys = csys;
        }
        const int ibase = ci * NB_CLUSTER + 4 * h;
        int v = stage_adj(p, s_st[warp][0], t0, t1, 0, lane);
        if (lane < 4) {
            const float4 x = p.xq[ibase + lane];
            s_xi[warp][lane] = make_float4(x.x, x.y, x.z, x.w * NB_COULOMB_F);
            s_gi[warp][lane] = p.gsort[ibase + lane];
            s_tr[warp][lane] = p.tsort[ibase + lane] * p.ntype;
        }
        float4 bi[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) bi[a] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int ngroups = (t1 - t0 + 3) >> 2;
        cp_async_wait_all();
        __syncwarp();
        for (int g = 0; g < ngroups; ++g) {
            const BvtStage &cs = s_st[warp][g & 1];
            const float4 xj = cs.xj[lane];
            const float4 gj = cs.gj[lane];
            const int tj = cs.tj[lane];
            const unsigned mrow = cs.m[lane] >> (lane & 7);
            const float4 S = s_shift[warp][(unsigned)v >> 27];
            const int slot = v & 0x07ffffff;
            const float qj_f = xj.w * NB_COULOMB_F;
            float4 bj = make_float4(0.f, 0.f, 0.f, 0.f);
            int vn = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (a == 2)  // next group's copies overlap rows 2 and 3 (past the last group: pad copies)
                    vn = stage_adj(p, s_st[warp][(g + 1) & 1], t0, t1, g + 1, lane);
                const float4 xi = s_xi[warp][a];
                float d6, d12;
                nb_pair_adj<true, COUL>(xi, xi.w, s_gi[warp][a], xj, qj_f, gj, s_lj[s_tr[warp][a] + tj], S.x, S.y, S.z,
                                  ((mrow >> (8 * a)) & 1u) != 0u, p.cc, p.k2, bi[a], bj, d6, d12);
                // the lane's own column: tj < ntype <= NT (the gather keeps types in range)
                acc[(a * NT + tj) * 2 + 0][lane] += d6;
                acc[(a * NT + tj) * 2 + 1][lane] += d12;
            }
            if (slot != p.pad_slot)  // all padding lanes share one slot: no atomics there
                atomicAdd(p.bsort + slot, bj);
            v = vn;
            cp_async_wait_all();
            __syncwarp();
        }
        // i side: value 4a + c (c = x, y, z, q); lane 8a then holds row a's x
        // and finds y, z, q 2, 4 and 6 lanes up
        {
            float r[16];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                r[4 * a + 0] = bi[a].x;
                r[4 * a + 1] = bi[a].y;
                r[4 * a + 2] = bi[a].z;
                r[4 * a + 3] = bi[a].w;
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
    const size_t smem = sizeof(float4) * (size_t)p.ntype * p.ntype;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward_vt<NT, COUL>, kBvtThreads,
                                                                      sizeof(float4) * 16);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    // small systems: each half's groups split into up to 8 ranges (one work item each)
    p.nseg = nb_work_split(pl->num_sms * per_sm * kBvtWarps, 2 * p.nreg * pl->nc_max);
    const int blocks = min(pl->num_sms * per_sm, (2 * p.nreg * pl->nc_max * p.nseg + kBvtWarps - 1) / kBvtWarps);
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
