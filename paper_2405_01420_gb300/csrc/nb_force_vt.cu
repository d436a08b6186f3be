// Force kernel over gathered tiles (the pruned list in its packed form).
//
// After a prune, each half i-cluster (rows 0-3 or 4-7 of an 8-atom cluster)
// has a list of 4 x 8 tiles whose 8 j atoms are gathered from all its
// cluster pairs: only j atoms within r_inner of at least one of the 4 rows
// appear, each with its own periodic shift. On water at rc 1.0 / r_inner
// 1.04 nm about 63% of the computed pair slots are in range, against 40% for
// 8 x 8 cluster tiles with empty half-tiles skipped; the arithmetic per pair
// is the same (nb_pair with d = (y_a - y_b) + S).
//
// One warp per half i-cluster; lane l owns i-row a = l >> 3 and tile column
// p = l & 7, i.e. mask bit l. Tiles are staged in shared memory CHUNK at a
// time (j coordinates, types, shift vectors, slots). j forces reduce-scatter
// over the 4 lanes of a column and are added with one atomic per (atom,
// component); i forces stay in registers for the whole half.
#include "nb_pair.cuh"

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
    float stale_prune2;
};

__device__ __forceinline__ void flush_energies_vt(double ec, double elj, int lane, double *out) {
    for (int o = 16; o > 0; o >>= 1) {
        ec += __shfl_xor_sync(0xffffffffu, ec, o);
        elj += __shfl_xor_sync(0xffffffffu, elj, o);
    }
    if (lane == 0 && out) {
        atomicAdd(&out[0], elj);
        atomicAdd(&out[1], ec);
    }
}

template <bool ENERGY, bool COUNT, int THREADS, int CHUNK>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_force_vt(VtParams p) {
    constexpr int kWarps = THREADS / 32;
    extern __shared__ float4 s_lj[];
    __shared__ unsigned s_mask[kWarps][CHUNK];
    __shared__ float4 s_xj[kWarps][CHUNK * 8];
    __shared__ float4 s_S[kWarps][CHUNK * 8];
    __shared__ int s_tj[kWarps][CHUNK * 8];
    __shared__ int s_slot[kWarps][CHUNK * 8];
    const int nt2 = p.ntype * p.ntype;
    for (int k = threadIdx.x; k < nt2; k += blockDim.x) {
        const float c6 = p.ljparams[2 * k], c12 = p.ljparams[2 * k + 1];
        s_lj[k] = make_float4(c6, c12, c12 * p.rc12inv - c6 * p.rc6inv, 0.0f);
    }
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
    const int pcol = lane & 7, a = lane >> 3;
    const unsigned lanebit = 1u << lane;
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    const int comp = (hi16 ? 2 : 0) + (hi8 ? 1 : 0);
    const unsigned nwork = 2u * (unsigned)p.st->nc;
    double ecd = 0.0, eljd = 0.0;
    int cur_sys = -1;
    unsigned cnt = 0;

    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&p.st->work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        const int ci = (w < nwork && p.order) ? p.order[w >> 1] : (int)(w >> 1);
        const int h = (int)(w & 1u);
        const int csys = (w < nwork) ? p.clus_sys[ci] : -1;
        if (ENERGY && csys != cur_sys) {
            if (cur_sys >= 0) flush_energies_vt(ecd, eljd, lane, p.energies + 2 * cur_sys);
            ecd = 0.0;
            eljd = 0.0;
            cur_sys = csys;
        }
        if (w >= nwork) break;
        const float4 *shift = p.sys_shift + 27 * csys;
        const int islot = ci * NB_CLUSTER + 4 * h + a;
        const float4 xi = p.xq[islot];
        const float qi = xi.w * NB_COULOMB_F;
        const int tr = p.tsort[islot] * p.ntype;
        const int t0 = p.half_start[2 * ci + h], t1 = t0 + p.half_len[2 * ci + h];
        float3 fi = make_float3(0.f, 0.f, 0.f);
        float ec = 0.0f, ecomp = 0.0f, elj = 0.0f, eljcomp = 0.0f;
        for (int base = t0; base < t1; base += CHUNK) {
            const int nch = min(CHUNK, t1 - base);
            __syncwarp();
            if (lane < nch) s_mask[warp][lane] = p.vt_mask[base + lane];
            for (int idx = lane; idx < nch * 8; idx += 32) {
                const int v = p.vt_slot[8 * (size_t)base + idx];
                const int slot = v & 0x07ffffff;
                s_slot[warp][idx] = slot;
                s_xj[warp][idx] = p.xq[slot];
                s_tj[warp][idx] = p.tsort[slot];
                s_S[warp][idx] = shift[(unsigned)v >> 27];
            }
            __syncwarp();
            for (int t = 0; t < nch; ++t) {
                const unsigned m = s_mask[warp][t];
                const int jdx = t * 8 + pcol;
                const float4 xj = s_xj[warp][jdx];
                const float4 S = s_S[warp][jdx];
                const int tj = s_tj[warp][jdx];
                float3 fj = make_float3(0.f, 0.f, 0.f);
                float ect = 0.0f, eljt = 0.0f;
                const int c1 = nb_pair<true, ENERGY>(xi, qi, xj, s_lj[tr + tj], S.x, S.y, S.z, (m & lanebit) != 0u,
                                                     p.cc, fi, fj, ect, eljt);
                if (COUNT) cnt += c1;
                float ka = hi16 ? fj.z : fj.x, sa = hi16 ? fj.x : fj.z;
                float kb = hi16 ? 0.0f : fj.y, sb = hi16 ? fj.y : 0.0f;
                ka += __shfl_xor_sync(0xffffffffu, sa, 16);
                kb += __shfl_xor_sync(0xffffffffu, sb, 16);
                float kk = hi8 ? kb : ka, ss = hi8 ? ka : kb;
                kk += __shfl_xor_sync(0xffffffffu, ss, 8);
                if (comp < 3) atomicAdd(p.fsort + 4 * s_slot[warp][jdx] + comp, kk);
                if (ENERGY) {
                    const float y = ect - ecomp;
                    const float tt = ec + y;
                    ecomp = (tt - ec) - y;
                    ec = tt;
                    const float yl = eljt - eljcomp;
                    const float tl = elj + yl;
                    eljcomp = (tl - elj) - yl;
                    elj = tl;
                }
            }
        }
        // i forces: sum over the 8 lanes of a row, lane p < 3 adds component p
        for (int o = 1; o < 8; o <<= 1) {
            fi.x += __shfl_xor_sync(0xffffffffu, fi.x, o);
            fi.y += __shfl_xor_sync(0xffffffffu, fi.y, o);
            fi.z += __shfl_xor_sync(0xffffffffu, fi.z, o);
        }
        if (pcol < 3) atomicAdd(p.fsort + 4 * islot + pcol, pcol == 0 ? fi.x : (pcol == 1 ? fi.y : fi.z));
        if (ENERGY) {
            ecd += (double)ec - (double)ecomp;
            eljd += (double)elj - (double)eljcomp;
        }
    }
    if (COUNT) {
        unsigned long long c64 = cnt;
        for (int o = 16; o > 0; o >>= 1) c64 += __shfl_xor_sync(0xffffffffu, c64, o);
        if (lane == 0) atomicAdd(&p.st->npairs, c64);
    }
}

using VtFn = void (*)(VtParams);
template <bool E, bool C>
VtFn pick_vt(int threads, int chunk) {
    if (threads == 128) return chunk == 8 ? k_force_vt<E, C, 128, 8> : k_force_vt<E, C, 128, 16>;
    return chunk == 8 ? k_force_vt<E, C, 256, 8> : k_force_vt<E, C, 256, 16>;
}

int g_vt_blocks_per_sm[2][2][2][2] = {};

}  // namespace

cudaError_t nb_launch_force_vt(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                               double *energies, float stale_prune2, cudaStream_t s) {
    VtParams p;
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
    p.cc.rc2 = rc * rc;
    p.cc.beta = beta;
    p.cc.kexp = (float)(-(double)beta * beta * 1.4426950408889634);
    p.cc.c2b = (float)(2.0 * beta / 1.7724538509055159);
    p.stale_prune2 = stale_prune2;
    const int e = energies ? 1 : 0;
    const int c = (pl->flags & NB_FLAG_COUNT_PAIRS) ? 1 : 0;
    const int threads = pl->force_threads == 128 ? 128 : 256;
    const int chunk = pl->force_chunk == 8 ? 8 : 16;
    VtFn fn = e ? (c ? pick_vt<true, true>(threads, chunk) : pick_vt<true, false>(threads, chunk))
                : (c ? pick_vt<false, true>(threads, chunk) : pick_vt<false, false>(threads, chunk));
    const size_t smem = sizeof(float4) * (size_t)ntype * ntype;
    int &per_sm = g_vt_blocks_per_sm[e][c][threads == 128][chunk == 8];
    if (per_sm == 0) {
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, (const void *)fn, threads, sizeof(float4) * NB_MAX_TYPES * NB_MAX_TYPES);
        if (err != cudaSuccess) return err;
        if (per_sm < 1) per_sm = 1;
    }
    const int use = pl->force_blocks_per_sm > 0 ? min(pl->force_blocks_per_sm, per_sm) : per_sm;
    int blocks = pl->num_sms * use;
    blocks = min(blocks, (2 * pl->nc_max + threads / 32 - 1) / (threads / 32));
    fn<<<max(blocks, 1), threads, smem, s>>>(p);
    return cudaGetLastError();
}
