// Adjoint of the force kernel (the "differentiation" form of the path):
// given g = dL/dF, the gradients of L with respect to positions, charges
// and the LJ C6/C12 matrix, recomputing every pair term over the same list.
//
// Per pair (d = y_a - y_b + S, F_a += s d, F_b -= s d) with u = g_a - g_b:
//   dL/dx_a += s u + (s'/r)(u.d) d          dL/dx_b -= the same
//   dL/dq_a += f q_b B (u.d)                dL/dq_b += f q_a B (u.d)
//   dL/dC6  += -6 r^-8 (u.d),  dL/dC12 += 12 r^-14 (u.d)   (type pair of a, b)
// with B = [erfc(beta r)/r + (2 beta/sqrt(pi)) exp(-beta^2 r^2)] / r^2 and
//   s'/r = [-3 s_C - 2 f q_a q_b (2 beta/sqrt(pi)) beta^2 exp(-beta^2 r^2)
//           + (48 C6/r^6 - 168 C12/r^12)/r^2] / r^2.
// The LJ gradient is reported for the symmetric matrix: each type pair's
// derivative is split evenly between (ti, tj) and (tj, ti).
//
// k_gather_g   g (original order) -> gsort (cluster order); zeroes the
//              gradient accumulators.
// k_backward   (8 x 8 cluster tiles; after a prune the gathered-tile form in
//              nb_backward_vt.cu runs instead)
//              one warp per i-cluster (work counter), list entries and their
//              j data staged in shared memory, lane layout as in k_force;
//              j-side gradients (x, y, z, q) reduce-scatter so every lane adds
//              one component; per-lane LJ accumulators by j type (NT <= 4).
// k_bwd_final  symmetrises the FP64 LJ accumulators into the output.
// k_bwd_scatter  cluster order -> original order.
#include "nb_pair.cuh"

namespace {

constexpr int kBwdThreads = 256;
constexpr int kBwdWarps = kBwdThreads / 32;
constexpr int kChunk = 16;

struct BwdParams {
    const float4 *xq;
    const int *tsort;
    const float4 *gsort;
    float *bsort;     // float4 per slot (dx, dy, dz, dq), viewed as floats
    double *glj_acc;  // [ntype][ntype][2] unsymmetrised, FP64
    const int4 *list;
    const int *ci_start;
    const int *ci_len;
    const int *order;  // i-clusters by decreasing list length, or NULL
    const float *ljparams;
    nb_dev_state *st;
    const float4 *sys_shift;  // [27 nsys]
    const int *clus_sys;
    int ntype;
    nb_coul cc;
    float k2;  // 2 (2 beta/sqrt(pi)) beta^2
    float stale_search2, stale_prune2;
    int has_inner;
};

__global__ void k_gather_g(int nmax_slots, const int *__restrict__ perm, const float *__restrict__ g,
                           float4 *__restrict__ gsort, float4 *__restrict__ bsort, double *__restrict__ glj_acc,
                           int nlj, const nb_dev_state *st) {
    nb_pdl_wait();
    nb_pdl_release();
    const int nslot = min(st->nc * NB_CLUSTER, nmax_slots);
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < nslot; slot += gridDim.x * blockDim.x) {
        const int atom = perm[slot];
        gsort[slot] = atom < 0 ? make_float4(0.f, 0.f, 0.f, 0.f)
                               : make_float4(g[3 * atom], g[3 * atom + 1], g[3 * atom + 2], 0.f);
        bsort[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < nlj; k += blockDim.x) glj_acc[k] = 0.0;
}

template <int NT>
__device__ __forceinline__ void add_onehot(float (&acc)[NT][2], const int tj, const float d6, const float d12) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float oh = (tj == t) ? 1.0f : 0.0f;
        acc[t][0] = fmaf(oh, d6, acc[t][0]);
        acc[t][1] = fmaf(oh, d12, acc[t][1]);
    }
}

template <int NT, int COUL>
__global__ void __launch_bounds__(kBwdThreads) k_backward(BwdParams p) {
    extern __shared__ float4 s_lj[];
    __shared__ int4 s_ent[kBwdWarps][kChunk];
    __shared__ float4 s_xj[kBwdWarps][kChunk * NB_CLUSTER];
    __shared__ float4 s_gj[kBwdWarps][kChunk * NB_CLUSTER];
    __shared__ int s_tj[kBwdWarps][kChunk * NB_CLUSTER];
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
        if (!p.has_inner && __uint_as_float(ds) > p.stale_search2) atomicOr(&p.st->err, NB_DEV_STALE_SEARCH);
        if (p.has_inner && __uint_as_float(dp) > p.stale_prune2) atomicOr(&p.st->err, NB_DEV_STALE_PRUNE);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = lane & 7, a1 = lane >> 3, a2 = a1 + 4;
    const unsigned lanebit = 1u << lane;
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    const int comp = (hi16 ? 2 : 0) + (hi8 ? 1 : 0);
    int4 *ent = s_ent[warp];
    float4 *sxj = s_xj[warp];
    float4 *sgj = s_gj[warp];
    int *stj = s_tj[warp];
    const int nc = p.st->nc;

    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&p.st->work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= (unsigned)nc) break;
        const int ci = p.order ? p.order[w] : (int)w;
        const float4 *shift = p.sys_shift + 27 * p.clus_sys[ci];
        const int k0 = p.ci_start[ci], k1 = k0 + p.ci_len[ci];
        const float4 xi1 = p.xq[ci * NB_CLUSTER + a1], xi2 = p.xq[ci * NB_CLUSTER + a2];
        const float4 gi1 = p.gsort[ci * NB_CLUSTER + a1], gi2 = p.gsort[ci * NB_CLUSTER + a2];
        const float qi1 = xi1.w * NB_COULOMB_F, qi2 = xi2.w * NB_COULOMB_F;
        const int ti1 = p.tsort[ci * NB_CLUSTER + a1], ti2 = p.tsort[ci * NB_CLUSTER + a2];
        const int tr1 = ti1 * p.ntype, tr2 = ti2 * p.ntype;
        float4 bi1 = make_float4(0.f, 0.f, 0.f, 0.f), bi2 = make_float4(0.f, 0.f, 0.f, 0.f);
        float acc1[NT][2], acc2[NT][2];
#pragma unroll
        for (int t = 0; t < NT; ++t) acc1[t][0] = acc1[t][1] = acc2[t][0] = acc2[t][1] = 0.0f;

        for (int base = k0; base < k1; base += kChunk) {
            const int nch = min(kChunk, k1 - base);
            __syncwarp();
            if (lane < nch) ent[lane] = p.list[base + lane];
            __syncwarp();
            for (int idx = lane; idx < nch * NB_CLUSTER; idx += 32) {
                const int slot = ent[idx >> 3].x * NB_CLUSTER + (idx & 7);
                sxj[idx] = p.xq[slot];
                sgj[idx] = p.gsort[slot];
                stj[idx] = p.tsort[slot];
            }
            __syncwarp();
            for (int t = 0; t < nch; ++t) {
                const int4 e = ent[t];
                const float4 xj = sxj[t * NB_CLUSTER + b];
                const float4 gj = sgj[t * NB_CLUSTER + b];
                const int tj = stj[t * NB_CLUSTER + b];
                const float qj_f = xj.w * NB_COULOMB_F;
                const unsigned mlo = (unsigned)e.z, mhi = (unsigned)e.w;
                float4 bj = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 S = shift[e.y];
                float d6, d12;
                if (mlo) {
                    if (e.y == NB_SHIFT_CENTER)
                        nb_pair_adj<false, COUL>(xi1, qi1, gi1, xj, qj_f, gj, s_lj[tr1 + tj], 0.f, 0.f, 0.f,
                                           (mlo & lanebit) != 0u, p.cc, p.k2, bi1, bj, d6, d12);
                    else
                        nb_pair_adj<true, COUL>(xi1, qi1, gi1, xj, qj_f, gj, s_lj[tr1 + tj], S.x, S.y, S.z,
                                          (mlo & lanebit) != 0u, p.cc, p.k2, bi1, bj, d6, d12);
                    add_onehot<NT>(acc1, tj, d6, d12);
                }
                if (mhi) {
                    if (e.y == NB_SHIFT_CENTER)
                        nb_pair_adj<false, COUL>(xi2, qi2, gi2, xj, qj_f, gj, s_lj[tr2 + tj], 0.f, 0.f, 0.f,
                                           (mhi & lanebit) != 0u, p.cc, p.k2, bi2, bj, d6, d12);
                    else
                        nb_pair_adj<true, COUL>(xi2, qi2, gi2, xj, qj_f, gj, s_lj[tr2 + tj], S.x, S.y, S.z,
                                          (mhi & lanebit) != 0u, p.cc, p.k2, bi2, bj, d6, d12);
                    add_onehot<NT>(acc2, tj, d6, d12);
                }
                // reduce-scatter (x, y, z, q) over the 4 lanes sharing b
                float ka = hi16 ? bj.z : bj.x, sa = hi16 ? bj.x : bj.z;
                float kb = hi16 ? bj.w : bj.y, sb = hi16 ? bj.y : bj.w;
                ka += __shfl_xor_sync(0xffffffffu, sa, 16);
                kb += __shfl_xor_sync(0xffffffffu, sb, 16);
                float kk = hi8 ? kb : ka, ss = hi8 ? ka : kb;
                kk += __shfl_xor_sync(0xffffffffu, ss, 8);
                atomicAdd(p.bsort + 4 * (e.x * NB_CLUSTER + b) + comp, kk);
            }
        }
        // i side: sum over the 8 lanes of a row (b varies), then lane b adds
        // component b & 3 of atom a1 (b < 4) or a2 (b >= 4)
        for (int o = 1; o < 8; o <<= 1) {
            bi1.x += __shfl_xor_sync(0xffffffffu, bi1.x, o);
            bi1.y += __shfl_xor_sync(0xffffffffu, bi1.y, o);
            bi1.z += __shfl_xor_sync(0xffffffffu, bi1.z, o);
            bi1.w += __shfl_xor_sync(0xffffffffu, bi1.w, o);
            bi2.x += __shfl_xor_sync(0xffffffffu, bi2.x, o);
            bi2.y += __shfl_xor_sync(0xffffffffu, bi2.y, o);
            bi2.z += __shfl_xor_sync(0xffffffffu, bi2.z, o);
            bi2.w += __shfl_xor_sync(0xffffffffu, bi2.w, o);
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                acc1[t][0] += __shfl_xor_sync(0xffffffffu, acc1[t][0], o);
                acc1[t][1] += __shfl_xor_sync(0xffffffffu, acc1[t][1], o);
                acc2[t][0] += __shfl_xor_sync(0xffffffffu, acc2[t][0], o);
                acc2[t][1] += __shfl_xor_sync(0xffffffffu, acc2[t][1], o);
            }
        }
        {
            const float4 bsel = b < 4 ? bi1 : bi2;
            const int c = b & 3;
            const float v = c == 0 ? bsel.x : (c == 1 ? bsel.y : (c == 2 ? bsel.z : bsel.w));
            atomicAdd(p.bsort + 4 * (ci * NB_CLUSTER + (b < 4 ? a1 : a2)) + c, v);
        }
        if (b == 0) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (t < p.ntype) {
                    atomicAdd(&p.glj_acc[2 * (tr1 + t)], (double)acc1[t][0]);
                    atomicAdd(&p.glj_acc[2 * (tr1 + t) + 1], (double)acc1[t][1]);
                    atomicAdd(&p.glj_acc[2 * (tr2 + t)], (double)acc2[t][0]);
                    atomicAdd(&p.glj_acc[2 * (tr2 + t) + 1], (double)acc2[t][1]);
                }
            }
        }
    }
}

__global__ void k_bwd_final(int ntype, const double *__restrict__ acc, double *__restrict__ out) {
    nb_pdl_wait();
    nb_pdl_release();
    const int k = threadIdx.x;
    if (k >= ntype * ntype) return;
    const int a = k / ntype, c = k % ntype;
    const int kt = c * ntype + a;
    out[2 * k] = 0.5 * (acc[2 * k] + acc[2 * kt]);
    out[2 * k + 1] = 0.5 * (acc[2 * k + 1] + acc[2 * kt + 1]);
}

__global__ void k_bwd_scatter(int n, const int *__restrict__ pos, const float4 *__restrict__ bsort,
                              float *__restrict__ grad_x, float *__restrict__ grad_q) {
    nb_pdl_wait();
    nb_pdl_release();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = bsort[pos[i]];
    grad_x[3 * i + 0] = v.x;
    grad_x[3 * i + 1] = v.y;
    grad_x[3 * i + 2] = v.z;
    grad_q[i] = v.w;
}

template <int NT, int COUL>
cudaError_t launch_bwd(nb_pairlist *pl, const BwdParams &p, cudaStream_t s) {
    const size_t smem = sizeof(float4) * (size_t)p.ntype * p.ntype;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward<NT, COUL>, kBwdThreads,
                                                                      sizeof(float4) * 16);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    int blocks = min(pl->num_sms * per_sm, (pl->nc_max + kBwdWarps - 1) / kBwdWarps);
    const cudaError_t e = nb_launch_pdl(k_backward<NT, COUL>, max(blocks, 1), kBwdThreads, smem, s, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int COUL>
cudaError_t launch_bwd_nt(nb_pairlist *pl, const BwdParams &p, cudaStream_t s) {
    if (p.ntype == 1) return launch_bwd<1, COUL>(pl, p, s);
    if (p.ntype == 2) return launch_bwd<2, COUL>(pl, p, s);
    return launch_bwd<4, COUL>(pl, p, s);
}

}  // namespace

cudaError_t nb_launch_backward(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                               const float *g, float *grad_x, float *grad_q, double *grad_lj,
                               float stale_search2, float stale_prune2, cudaStream_t s) {
    const int nslot = pl->nc_max * NB_CLUSTER;
    const int nlj = 2 * ntype * ntype;
    int gb = min((nslot + 255) / 256, pl->num_sms * 8);
    cudaError_t e = nb_launch_pdl(k_gather_g, max(gb, 1), 256, 0, s, nslot, (const int *)pl->perm, g, pl->gsort,
                                  pl->bsort, pl->glj_acc, nlj, (const nb_dev_state *)pl->st);
    if (e != cudaSuccess) return e;
    BwdParams p;
    p.xq = pl->xq;
    p.tsort = pl->tsort;
    p.gsort = pl->gsort;
    p.bsort = reinterpret_cast<float *>(pl->bsort);
    p.glj_acc = pl->glj_acc;
    p.list = pl->has_inner ? pl->inner : pl->outer;
    p.ci_start = pl->ci_start;
    p.ci_len = pl->has_inner ? pl->ci_len_inner : pl->ci_len_outer;
    p.order = pl->sorted ? pl->ci_order : nullptr;
    p.ljparams = ljparams;
    p.st = pl->st;
    p.sys_shift = pl->sys_shift;
    p.clus_sys = pl->clus_sys;
    p.ntype = ntype;
    const int coul = nb_fill_coul(p.cc, rc, beta, pl->coul_kind, pl->eps_rf, pl->coul_flags);
    p.k2 = (float)(2.0 * (2.0 * beta / 1.7724538509055159) * (double)beta * beta);
    p.stale_search2 = stale_search2;
    p.stale_prune2 = stale_prune2;
    p.has_inner = pl->has_inner;
    if (pl->has_vtiles && !(pl->flags & NB_FLAG_CLUSTER_TILES))  // gathered tiles after a prune
        e = nb_launch_backward_vt(pl, ntype, ljparams, rc, beta, stale_prune2, s);
    else if (coul == NB_COULK_RF)  // the Ewald shift does not change forces
        e = launch_bwd_nt<NB_COULK_RF>(pl, p, s);
    else
        e = launch_bwd_nt<NB_COULK_EWALD>(pl, p, s);
    if (e != cudaSuccess) return e;
    if ((pl->coul_flags & NB_COUL_EXCL_CORR) && pl->has_excl) {
        e = nb_launch_excl_corr_adj(pl, rc, beta, s);
        if (e != cudaSuccess) return e;
    }
    e = nb_launch_pdl(k_bwd_final, 1, 32, 0, s, ntype, (const double *)pl->glj_acc, grad_lj);
    if (e != cudaSuccess) return e;
    const int n = pl->n_atoms;
    return nb_launch_pdl(k_bwd_scatter, (n + 255) / 256, 256, 0, s, n, (const int *)pl->pos, (const float4 *)pl->bsort,
                         grad_x, grad_q);
}
