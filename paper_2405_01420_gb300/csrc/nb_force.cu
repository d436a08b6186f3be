// Nonbonded forces and energies over the cluster-pair list (the NBNXM
// kernel of §III-A), plus the gather that feeds it and the permute-back
// that follows it.
//
// k_gather   coords/q/type (original order) -> xq (float4 y,q) / tsort in
//            cluster order; y is the image nearest the search-frame
//            position. Zeroes the force accumulators, tracks the largest
//            displacement since the search and since the last prune. The
//            prune's gather (snapshot) records the positions of the prune
//            and clears the list-length histogram the prune fills.
// k_force    persistent grid, one warp per i-cluster (each warp's first
//            from its grid index, later ones from a work counter). List entries and their j-cluster data are staged in
//            shared memory 16 at a time. Lane l owns j-atom b = l & 7 and i-atoms l >> 3 and
//            (l >> 3) + 4, i.e. exactly mask bits l (low word) and 32 + l
//            (high word). i-forces stay in registers for the whole list of
//            ci; j-forces are reduced across the four lanes sharing b with
//            a reduce-scatter (3 shuffles) and added with one atomic per
//            (atom, component) per 8x8 tile. Half-tiles (mask word 0) are
//            skipped by a warp-uniform branch. Energies: per-lane FP32 per
//            tile, Kahan-compensated across tiles, FP64 per
//            i-cluster and across the grid.
// k_scatter  forces of cluster slots -> original atom order.
#include "nb_pair.cuh"

namespace {


struct GatherParams {
    const int *perm;
    const float *coords;
    const float *q;
    const int *type;
    const float4 *xref;
    float4 *xprune;
    float4 *xq;
    int *tsort;
    float4 *fsort;
    nb_dev_state *st;
    double *energies;  // [2 nsys] or NULL
    const nb_sys *sys;
    const int *clus_sys;
    int *len_hist;  // cleared here ahead of a prune that fills it, or NULL
    int nsys;
    int snapshot;
    int ntype;
    int part;    // NB_PART_ALL / NB_PART_LOCAL (home atoms) / NB_PART_NONLOCAL (halo atoms)
    int n_home;  // atoms [0, n_home) are home atoms
};

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(256) k_gather(GatherParams p) {
    nb_pdl_wait();
    nb_pdl_release();
    const int nslot = p.st->nc * NB_CLUSTER;
    float d2s_max = 0.0f, d2p_max = 0.0f;
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < nslot; slot += gridDim.x * blockDim.x) {
        const int atom = p.perm[slot];
        if (p.part != NB_PART_NONLOCAL) p.fsort[slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (atom < 0) continue;
        if (p.part == NB_PART_LOCAL ? atom >= p.n_home : (p.part == NB_PART_NONLOCAL && atom < p.n_home)) continue;
        const float4 r = p.xref[slot];
        const float4 L = p.sys[p.clus_sys[slot / NB_CLUSTER]].box;  // does not wait for perm
        float x = p.coords[3 * atom + 0], y = p.coords[3 * atom + 1], z = p.coords[3 * atom + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
            atomicOr(&p.st->err, NB_DEV_NONFINITE);
            x = r.x;
            y = r.y;
            z = r.z;
        }
        const float yx = nb_image(x, r.x, L.x), yy = nb_image(y, r.y, L.y), yz = nb_image(z, r.z, L.z);
        p.xq[slot] = make_float4(yx, yy, yz, p.q ? p.q[atom] : 0.0f);
        if (p.type) {
            int t = p.type[atom];
            if (t < 0 || t >= p.ntype) {  // keep the LJ table lookup in bounds
                atomicOr(&p.st->err, NB_DEV_BAD_TYPE);
                t = 0;
            }
            p.tsort[slot] = t;
        }
        float ex = yx - r.x, ey = yy - r.y, ez = yz - r.z;
        d2s_max = fmaxf(d2s_max, ex * ex + ey * ey + ez * ez);
        if (p.snapshot) {
            p.xprune[slot] = make_float4(yx, yy, yz, 0.0f);
        } else {
            const float4 pr = p.xprune[slot];
            ex = yx - pr.x;
            ey = yy - pr.y;
            ez = yz - pr.z;
            d2p_max = fmaxf(d2p_max, ex * ex + ey * ey + ez * ez);
        }
    }
    d2s_max = warp_max(d2s_max);
    d2p_max = warp_max(d2p_max);
    if ((threadIdx.x & 31) == 0) {
        // non-negative floats order like their bit patterns
        if (d2s_max > 0.0f) atomicMax(&p.st->cur_d2_search, __float_as_uint(d2s_max));
        if (d2p_max > 0.0f) atomicMax(&p.st->cur_d2_prune, __float_as_uint(d2p_max));
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            p.st->work = 0u;
            p.st->npairs = 0ull;
            if (p.snapshot) {  // a prune follows this gather
                p.st->work_prune = 0u;
                p.st->inner_count = 0ull;
                p.st->tile_count = 0ull;
                p.st->nl_count = 0u;
            }
        }
        if (p.energies && p.part != NB_PART_NONLOCAL)
            for (int k = threadIdx.x; k < 2 * p.nsys; k += blockDim.x) p.energies[k] = 0.0;
        if (p.len_hist)
            for (int k = threadIdx.x; k < NB_LEN_BINS; k += blockDim.x) p.len_hist[k] = 0;
    }
}

struct ForceParams {
    const float4 *xq;
    const int *tsort;
    float *fsort;  // float4 per slot, viewed as floats
    const int4 *list;
    const int *ci_start;
    const int *ci_len;
    const int *order;         // i-clusters by decreasing list length, or NULL
    const float *ljparams;
    nb_dev_state *st;
    double *energies;         // [2 nsys]
    const float4 *sys_shift;  // [27 nsys]
    const int *clus_sys;
    int ntype;
    float rc6inv, rc12inv;  // 1/rc^6, 1/rc^12 for the LJ potential shift
    nb_coul cc;
    float stale_search2, stale_prune2;
    int has_inner;
    int part;                        // NB_PART_*: ALL computes every pair
    const unsigned char *clus_home;  // with a part: bit b = slot b of the cluster holds a home atom
    int finalize;                    // move the displacement maxima of this evaluation to last_*
};


// Adds a warp's FP64 energy partials (E_LJ, E_C) of one system to out[0..1].
__device__ __forceinline__ void flush_energies(double ec, double elj, int lane, double *out) {
    for (int o = 16; o > 0; o >>= 1) {
        ec += __shfl_xor_sync(0xffffffffu, ec, o);
        elj += __shfl_xor_sync(0xffffffffu, elj, o);
    }
    if (lane == 0 && out) {
        atomicAdd(&out[0], elj);
        atomicAdd(&out[1], ec);
    }
}

// THREADS per block and CHUNK list entries staged per warp are launch
// shapes the autotuner chooses among (nb_set_force_shape); both keep the
// register cap at 80 (3 blocks of 256 or 6 of 128 threads per SM). At a cap
// of 64 (4 or 8 blocks) the kernel was 11% slower on the 96,000-atom list
// and the 1,536-atom force call 24.0 against 22.2 us.
template <bool ENERGY, bool COUNT, int THREADS, int CHUNK, int COUL>
__global__ void __launch_bounds__(THREADS, 768 / THREADS) k_force(ForceParams p) {
    constexpr int kWarps = THREADS / 32;
    extern __shared__ float4 s_lj[];  // ntype^2 entries (C6, C12, E shift, 0)
    __shared__ int4 s_ent[kWarps][CHUNK];
    __shared__ float4 s_xj[kWarps][CHUNK * NB_CLUSTER];
    __shared__ int s_tj[kWarps][CHUNK * NB_CLUSTER];
    __shared__ unsigned char s_hj[kWarps][CHUNK];  // home bits of the staged j clusters
    nb_pdl_wait();
    nb_pdl_release();
    const int nt2 = p.ntype * p.ntype;
    for (int k = threadIdx.x; k < nt2; k += blockDim.x) {
        const float c6 = p.ljparams[2 * k], c12 = p.ljparams[2 * k + 1];
        s_lj[k] = make_float4(c6, c12, c12 * p.rc12inv - c6 * p.rc6inv, 0.0f);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // The gather of this call has finished; record its displacements and
        // check them against the list buffers.
        const unsigned ds = p.st->cur_d2_search, dp = p.st->cur_d2_prune;
        if (p.finalize) {
            p.st->last_d2_search = ds;
            p.st->last_d2_prune = dp;
            p.st->cur_d2_search = 0u;
            p.st->cur_d2_prune = 0u;
        }
        if (!p.has_inner && __uint_as_float(ds) > p.stale_search2) atomicOr(&p.st->err, NB_DEV_STALE_SEARCH);
        if (p.has_inner && __uint_as_float(dp) > p.stale_prune2) atomicOr(&p.st->err, NB_DEV_STALE_PRUNE);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = lane & 7, a1 = lane >> 3, a2 = a1 + 4;
    const unsigned lanebit = 1u << lane;
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    const int comp = (hi16 ? 2 : 0) + (hi8 ? 1 : 0);  // component this lane adds after the reduce-scatter
    int4 *ent = s_ent[warp];
    float4 *sxj = s_xj[warp];
    int *stj = s_tj[warp];
    const int nc = p.st->nc;
    double ecd = 0.0, eljd = 0.0;  // energies of system cur_sys not yet added to the output
    int cur_sys = -1;
    unsigned cnt = 0;

    const unsigned nseg = nb_work_split(gridDim.x * kWarps, (unsigned)nc);
    const unsigned nwork = (unsigned)nc * nseg;
    const unsigned nwarps = gridDim.x * kWarps;
    for (unsigned it = 0;; ++it) {
        // a warp's first work item is its own index in the grid, later ones come from the
        // counter: thousands of warps do not start on one contended atomic
        unsigned w = blockIdx.x * kWarps + warp;
        if (it > 0) {
            unsigned a = 0;
            if (lane == 0) a = atomicAdd(&p.st->work, 1u);
            w = __shfl_sync(0xffffffffu, a, 0) + nwarps;
        }
        // work item w: range seg of the list of the i-cluster at position idx of the order
        const unsigned idx = nseg == 1u ? w : w / nseg, seg = w - idx * nseg;
        const int ci = (w < nwork && p.order) ? p.order[idx] : (int)idx;
        const int csys = (w < nwork) ? p.clus_sys[ci] : -1;
        if (ENERGY && csys != cur_sys) {
            if (cur_sys >= 0) flush_energies(ecd, eljd, lane, p.energies + 2 * cur_sys);
            ecd = 0.0;
            eljd = 0.0;
            cur_sys = csys;
        }
        if (w >= nwork) break;
        const float4 *shift = p.sys_shift + 27 * csys;
        const int kc = p.ci_start[ci];
        int r0, r1;
        nb_piece(p.ci_len[ci], seg, nseg, r0, r1);
        const int k0 = kc + r0, k1 = kc + r1;
        if (k1 <= k0) continue;
        const float4 xi1 = p.xq[ci * NB_CLUSTER + a1], xi2 = p.xq[ci * NB_CLUSTER + a2];
        const float qi1 = xi1.w * NB_COULOMB_F, qi2 = xi2.w * NB_COULOMB_F;
        const int tr1 = p.tsort[ci * NB_CLUSTER + a1] * p.ntype;
        const int tr2 = p.tsort[ci * NB_CLUSTER + a2] * p.ntype;
        const unsigned hci = p.part != NB_PART_ALL ? p.clus_home[ci] : 0u;
        const bool hi1 = (hci >> a1) & 1u, hi2 = (hci >> a2) & 1u;
        float3 fi1 = make_float3(0.0f, 0.0f, 0.0f), fi2 = make_float3(0.0f, 0.0f, 0.0f);
        float ec = 0.0f, ecomp = 0.0f, elj = 0.0f, eljcomp = 0.0f;

        for (int base = k0; base < k1; base += CHUNK) {
            // Stage up to CHUNK entries and their j-cluster coordinates and
            // types: independent, batched loads instead of one dependent
            // chain per tile.
            const int nch = min(CHUNK, k1 - base);
            __syncwarp();
            if (lane < nch) {
                ent[lane] = p.list[base + lane];
                if (p.part != NB_PART_ALL) s_hj[warp][lane] = p.clus_home[ent[lane].x];
            }
            __syncwarp();
            for (int idx = lane; idx < nch * NB_CLUSTER; idx += 32) {
                const int slot = ent[idx >> 3].x * NB_CLUSTER + (idx & 7);
                sxj[idx] = p.xq[slot];
                stj[idx] = p.tsort[slot];
            }
            __syncwarp();
            for (int t = 0; t < nch; ++t) {
                const int4 e = ent[t];
                const float4 xj = sxj[t * NB_CLUSTER + b];
                const int tj = stj[t * NB_CLUSTER + b];
                const int sidx = e.y;
                unsigned mlo = (unsigned)e.z, mhi = (unsigned)e.w;
                if (p.part != NB_PART_ALL) {  // keep the pairs of this part: both atoms home, or not
                    const bool hj = (s_hj[warp][t] >> b) & 1u;
                    const unsigned l1 = __ballot_sync(0xffffffffu, hi1 && hj);
                    const unsigned l2 = __ballot_sync(0xffffffffu, hi2 && hj);
                    mlo &= p.part == NB_PART_LOCAL ? l1 : ~l1;
                    mhi &= p.part == NB_PART_LOCAL ? l2 : ~l2;
                }
                float3 fj = make_float3(0.0f, 0.0f, 0.0f);
                float ect = 0.0f, eljt = 0.0f;
                int c1 = 0, c2 = 0;
                if (sidx == NB_SHIFT_CENTER) {
                    if (mlo) c1 = nb_pair<false, ENERGY, COUL>(xi1, qi1, xj, s_lj[tr1 + tj], 0.f, 0.f, 0.f,
                                                         (mlo & lanebit) != 0u, p.cc, fi1, fj, ect, eljt);
                    if (mhi) c2 = nb_pair<false, ENERGY, COUL>(xi2, qi2, xj, s_lj[tr2 + tj], 0.f, 0.f, 0.f,
                                                         (mhi & lanebit) != 0u, p.cc, fi2, fj, ect, eljt);
                } else {
                    const float4 S = shift[sidx];
                    if (mlo) c1 = nb_pair<true, ENERGY, COUL>(xi1, qi1, xj, s_lj[tr1 + tj], S.x, S.y, S.z,
                                                        (mlo & lanebit) != 0u, p.cc, fi1, fj, ect, eljt);
                    if (mhi) c2 = nb_pair<true, ENERGY, COUL>(xi2, qi2, xj, s_lj[tr2 + tj], S.x, S.y, S.z,
                                                        (mhi & lanebit) != 0u, p.cc, fi2, fj, ect, eljt);
                }
                if (COUNT) cnt += c1 + c2;
                // Reduce fj over the lanes l, l^8, l^16, l^24 (same b) as a
                // reduce-scatter: afterwards lane l holds component comp.
                float ka = hi16 ? fj.z : fj.x, sa = hi16 ? fj.x : fj.z;
                float kb = hi16 ? 0.0f : fj.y, sb = hi16 ? fj.y : 0.0f;
                ka += __shfl_xor_sync(0xffffffffu, sa, 16);
                kb += __shfl_xor_sync(0xffffffffu, sb, 16);
                float kk = hi8 ? kb : ka, ss = hi8 ? ka : kb;
                kk += __shfl_xor_sync(0xffffffffu, ss, 8);
                if (comp < 3) atomicAdd(p.fsort + 4 * (e.x * NB_CLUSTER + b) + comp, kk);
                if (ENERGY) {  // Kahan-compensated sums across the tiles of ci
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
        // i-forces: sum over the 8 lanes sharing a1 (b varies: xor 1, 2, 4)
        for (int o = 1; o < 8; o <<= 1) {
            fi1.x += __shfl_xor_sync(0xffffffffu, fi1.x, o);
            fi1.y += __shfl_xor_sync(0xffffffffu, fi1.y, o);
            fi1.z += __shfl_xor_sync(0xffffffffu, fi1.z, o);
            fi2.x += __shfl_xor_sync(0xffffffffu, fi2.x, o);
            fi2.y += __shfl_xor_sync(0xffffffffu, fi2.y, o);
            fi2.z += __shfl_xor_sync(0xffffffffu, fi2.z, o);
        }
        if (b < 3) {
            const float v = b == 0 ? fi1.x : (b == 1 ? fi1.y : fi1.z);
            atomicAdd(p.fsort + 4 * (ci * NB_CLUSTER + a1) + b, v);
        } else if (b < 6) {
            const float v = b == 3 ? fi2.x : (b == 4 ? fi2.y : fi2.z);
            atomicAdd(p.fsort + 4 * (ci * NB_CLUSTER + a2) + (b - 3), v);
        }
        if (ENERGY) {
            ecd += (double)ec - (double)ecomp;
            eljd += (double)elj - (double)eljcomp;
        }
    }

    // pair count: one atomic per warp, no block barrier, so a warp that runs
    // out of work leaves without waiting for the rest of its block (the
    // energies were flushed when the loop ended)
    if (COUNT) {
        unsigned long long c64 = cnt;
        for (int o = 16; o > 0; o >>= 1) c64 += __shfl_xor_sync(0xffffffffu, c64, o);
        if (lane == 0) atomicAdd(&p.st->npairs, c64);
    }
}

__global__ void k_clus_home(int nc_max, const int *__restrict__ perm, int n_home,
                            unsigned char *__restrict__ clus_home, const nb_dev_state *st) {
    const int nc = st->nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc_max; c += gridDim.x * blockDim.x) {
        unsigned bits = 0u;
        if (c < nc)
            for (int b = 0; b < NB_CLUSTER; ++b) {
                const int atom = perm[c * NB_CLUSTER + b];
                bits |= (atom >= 0 && atom < n_home ? 1u : 0u) << b;
            }
        clus_home[c] = (unsigned char)bits;
    }
}

__global__ void k_scatter(int n, const int *__restrict__ pos, const float4 *__restrict__ fsort,
                          float *__restrict__ forces) {
    nb_pdl_wait();
    nb_pdl_release();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 f = fsort[pos[i]];
    forces[3 * i + 0] = f.x;
    forces[3 * i + 1] = f.y;
    forces[3 * i + 2] = f.z;
}

// kernel variants: [energy][count][threads 128/256][chunk 8/16]
using ForceFn = void (*)(ForceParams);
template <bool E, bool C, int K>
ForceFn pick_shape(int threads, int chunk) {
    if (threads == 128) return chunk == 8 ? k_force<E, C, 128, 8, K> : k_force<E, C, 128, 16, K>;
    return chunk == 8 ? k_force<E, C, 256, 8, K> : k_force<E, C, 256, 16, K>;
}

template <bool E, bool C>
ForceFn pick(int threads, int chunk, int coul) {
    if (coul == NB_COULK_RF) return pick_shape<E, C, NB_COULK_RF>(threads, chunk);
    if (coul == NB_COULK_EWALD_SHIFT) return pick_shape<E, C, NB_COULK_EWALD_SHIFT>(threads, chunk);
    return pick_shape<E, C, NB_COULK_EWALD>(threads, chunk);
}

int g_blocks_per_sm[3][2][2][2][2] = {};

}  // namespace

cudaError_t nb_launch_gather(nb_pairlist *pl, const float *coords, const float *q, const int *type,
                             int ntype, int snapshot, double *energies, int part, cudaStream_t s) {
    GatherParams p;
    p.part = part;
    p.n_home = pl->n_home;
    p.ntype = ntype;
    p.perm = pl->perm;
    p.coords = coords;
    p.q = q;
    p.type = type;
    p.xref = pl->xref;
    p.xprune = pl->xprune;
    p.xq = pl->xq;
    p.tsort = pl->tsort;
    p.fsort = pl->fsort;
    p.st = pl->st;
    p.energies = energies;
    p.sys = pl->sys;
    p.clus_sys = pl->clus_sys;
    p.len_hist = (snapshot && !(pl->flags & NB_FLAG_NO_LIST_SORT)) ? pl->len_hist : nullptr;
    p.nsys = pl->nsys;
    p.snapshot = snapshot;
    int blocks = (pl->nc_max * NB_CLUSTER + 255) / 256;
    blocks = max(1, min(blocks, pl->num_sms * 8));
    return nb_launch_pdl(k_gather, blocks, 256, 0, s, p);
}

cudaError_t nb_launch_force(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                            double *energies, float stale_search2, float stale_prune2, int part,
                            cudaStream_t s) {
    ForceParams p;
    p.part = part;
    p.clus_home = pl->clus_home;
    p.finalize = part != NB_PART_LOCAL;
    p.xq = pl->xq;
    p.tsort = pl->tsort;
    p.fsort = reinterpret_cast<float *>(pl->fsort);
    p.list = pl->has_inner ? pl->inner : pl->outer;
    p.ci_start = pl->ci_start;
    p.ci_len = pl->has_inner ? pl->ci_len_inner : pl->ci_len_outer;
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
    p.stale_search2 = stale_search2;
    p.stale_prune2 = stale_prune2;
    p.has_inner = pl->has_inner;
    const int e = energies ? 1 : 0;
    const int c = (pl->flags & NB_FLAG_COUNT_PAIRS) ? 1 : 0;
    const int threads = pl->force_threads == 128 ? 128 : 256;
    const int chunk = pl->force_chunk == 8 ? 8 : 16;
    ForceFn fn = e ? (c ? pick<true, true>(threads, chunk, coul) : pick<true, false>(threads, chunk, coul))
                   : (c ? pick<false, true>(threads, chunk, coul) : pick<false, false>(threads, chunk, coul));
    const size_t smem = sizeof(float4) * (size_t)ntype * ntype;
    int &per_sm = g_blocks_per_sm[coul][e][c][threads == 128][chunk == 8];
    if (per_sm == 0) {
        // occupancy at the largest LJ table, so that the grid never exceeds residency
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, (const void *)fn, threads, sizeof(float4) * NB_MAX_TYPES * NB_MAX_TYPES);
        if (err != cudaSuccess) return err;
        if (per_sm < 1) per_sm = 1;
    }
    int use = pl->force_blocks_per_sm > 0 ? min(pl->force_blocks_per_sm, per_sm) : per_sm;
    int blocks = pl->num_sms * use;
    // no more blocks than work items: at most NB_MAX_SPLIT per i-cluster
    blocks = min(blocks, (pl->nc_max * NB_MAX_SPLIT + threads / 32 - 1) / (threads / 32));
    blocks = max(blocks, 1);
    return nb_launch_pdl(fn, blocks, threads, smem, s, p);
}

cudaError_t nb_launch_clus_home(nb_pairlist *pl, cudaStream_t s) {
    const int blocks = max(1, min((pl->nc_max + 255) / 256, pl->num_sms * 8));
    k_clus_home<<<blocks, 256, 0, s>>>(pl->nc_max, pl->perm, pl->n_home, pl->clus_home, pl->st);
    return cudaGetLastError();
}

cudaError_t nb_launch_scatter(nb_pairlist *pl, float *forces, cudaStream_t s) {
    const int n = pl->n_atoms;
    return nb_launch_pdl(k_scatter, (n + 255) / 256, 256, 0, s, n, (const int *)pl->pos, (const float4 *)pl->fsort,
                         forces);
}
