// Cluster-pair search: the outer ("buffered") pair list at radius rlist
// (§III-A: "pair list buffer", "list range").
//
// One warp per i-cluster ci. The warp walks the grid columns whose xy extent
// lies within rlist of ci's bounding box (with periodic images), and in each
// column tests the clusters cj >= ci, one per lane, by bounding-box distance.
// Kept pairs get a shift index and a 64-bit mask (bit a*8+b: atom a of ci
// with atom b of cj) of real, non-excluded, non-duplicated atom pairs. The
// warp collects its entries in shared memory, reserves space in the list
// with one atomic, and writes them out coalesced.
//
// Half list: (ci, cj, S) and (cj, ci, -S) are the same interactions, so only
// cj >= ci is kept; for cj == ci the shift S = 0 keeps b > a and of each
// pair S, -S only the one with the larger shift index is kept.
#include "nb_internal.cuh"

namespace {

constexpr int kSearchWarps = 8;
// bit a*8+b set for b > a: each pair of one cluster with itself once
constexpr unsigned long long kUpperStrict = 0x0080C0E0F0F8FCFEull;
// bit a*8+a: an atom with its own periodic image
constexpr unsigned long long kDiagonal = 0x8040201008040201ull;

struct SearchParams {
    const float4 *bbox;
    const int *col_clus_start;
    const int *perm;
    const int *pos;
    const int *excl_off;
    const int *excl_idx;
    int4 *outer;
    int *ci_start;
    int *ci_len;
    int *ci_len_inner;
    nb_dev_state *st;
    const nb_sys *sys;
    const int *clus_sys;
    int n_atoms;
    float rl2;     // squared radius of the bounding-box test (already inflated)
    float rl_col;  // radius of the column / z-image pre-selection (inflated further)
    unsigned long long cap;
};

__device__ __forceinline__ unsigned long long row_mask(int n_real) {
    const unsigned long long ones = 0x0101010101010101ull;
    return n_real >= 8 ? ones : (ones & ((1ull << (8 * n_real)) - 1ull));
}

__device__ __forceinline__ int image_of(int ju, int n) { return ju < 0 ? -1 : (ju >= n ? 1 : 0); }

__global__ void __launch_bounds__(kSearchWarps * 32) k_search(SearchParams p) {
    extern __shared__ int4 s_entries[];  // kSearchWarps * NB_CI_ENTRY_BUF
    __shared__ int2 s_excl[kSearchWarps][NB_CI_EXCL_BUF];
    __shared__ int s_nexcl[kSearchWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int4 *buf = s_entries + warp * NB_CI_ENTRY_BUF;
    const int nc = p.st->nc;

    for (int ci = blockIdx.x * kSearchWarps + warp; ci < nc; ci += gridDim.x * kSearchWarps) {
        const float4 lo = p.bbox[2 * ci], hi = p.bbox[2 * ci + 1];
        const int ni = __float_as_int(lo.w);
        const nb_sys S = p.sys[p.clus_sys[ci]];  // every candidate column belongs to this system

        // exclusions of the i-atoms: (row a, slot of the excluded partner)
        if (lane == 0) s_nexcl[warp] = 0;
        __syncwarp();
        if (p.excl_off != nullptr && lane < ni) {
            int atom = p.perm[ci * NB_CLUSTER + lane];
            int k0 = p.excl_off[atom], k1 = p.excl_off[atom + 1];
            for (int k = k0; k < k1; ++k) {
                const int partner = p.excl_idx[k];
                if (partner < 0 || partner >= p.n_atoms) {  // keep the lookup in bounds
                    atomicOr(&p.st->err, NB_DEV_EXCL_OVERFLOW);
                    continue;
                }
                int ps = p.pos[partner];
                int idx = atomicAdd(&s_nexcl[warp], 1);
                if (idx < NB_CI_EXCL_BUF) s_excl[warp][idx] = make_int2(lane, ps);
            }
        }
        __syncwarp();
        int nex = s_nexcl[warp];
        if (nex > NB_CI_EXCL_BUF) {
            if (lane == 0) atomicOr(&p.st->err, NB_DEV_EXCL_OVERFLOW);
            nex = NB_CI_EXCL_BUF;
        }

        int nout = 0;
        int jx0 = max((int)floorf((lo.x - p.rl_col) * S.inv_sx), -S.ncx);
        int jx1 = min((int)floorf((hi.x + p.rl_col) * S.inv_sx), 2 * S.ncx - 1);
        int jy0 = max((int)floorf((lo.y - p.rl_col) * S.inv_sy), -S.ncy);
        int jy1 = min((int)floorf((hi.y + p.rl_col) * S.inv_sy), 2 * S.ncy - 1);
        for (int jxu = jx0; jxu <= jx1; ++jxu) {
            const int kx = image_of(jxu, S.ncx);
            const int jx = jxu - kx * S.ncx;
            const float ox = (float)kx * S.box.x;  // j image at x_b + ox, i.e. S_x = -ox
            for (int jyu = jy0; jyu <= jy1; ++jyu) {
                const int ky = image_of(jyu, S.ncy);
                const int jy = jyu - ky * S.ncy;
                const float oy = (float)ky * S.box.y;
                const int col = S.col_off + jx * S.ncy + jy;
                const int c0 = p.col_clus_start[col], c1 = p.col_clus_start[col + 1];
                if (c1 <= ci) continue;  // every cluster of this column precedes ci
                const int cs = max(c0, ci);
                for (int kz = -1; kz <= 1; ++kz) {
                    const float oz = (float)kz * S.box.z;
                    if (lo.z - p.rl_col > oz + S.box.z || hi.z + p.rl_col < oz) continue;
                    const int sidx = (1 - kx) * 9 + (1 - ky) * 3 + (1 - kz);
                    for (int cb = cs; cb < c1; cb += 32) {
                        const int c = cb + lane;
                        bool keep = false;
                        unsigned long long m = 0;
                        if (c < c1) {
                            const float4 bl = p.bbox[2 * c], bh = p.bbox[2 * c + 1];
                            float gx = fmaxf(0.0f, fmaxf((bl.x + ox) - hi.x, lo.x - (bh.x + ox)));
                            float gy = fmaxf(0.0f, fmaxf((bl.y + oy) - hi.y, lo.y - (bh.y + oy)));
                            float gz = fmaxf(0.0f, fmaxf((bl.z + oz) - hi.z, lo.z - (bh.z + oz)));
                            keep = gx * gx + gy * gy + gz * gz < p.rl2;
                            if (c == ci && sidx < NB_SHIFT_CENTER) keep = false;
                            if (keep) {
                                const int nj = __float_as_int(bl.w);
                                m = row_mask(ni) * (unsigned long long)((1u << nj) - 1u);
                                if (c == ci) m &= (sidx == NB_SHIFT_CENTER) ? kUpperStrict : ~kDiagonal;
                                for (int e = 0; e < nex; ++e) {
                                    const int2 ex = s_excl[warp][e];
                                    if ((ex.y >> 3) == c) m &= ~(1ull << (ex.x * 8 + (ex.y & 7)));
                                }
                                keep = (m != 0ull);
                            }
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, keep);
                        if (keep) {
                            const int r = nout + __popc(bal & ((1u << lane) - 1u));
                            if (r < NB_CI_ENTRY_BUF)
                                buf[r] = make_int4(c, sidx, (int)(unsigned)(m & 0xffffffffu),
                                                   (int)(unsigned)(m >> 32));
                        }
                        nout += __popc(bal);
                    }
                }
            }
        }
        if (nout > NB_CI_ENTRY_BUF) {
            if (lane == 0) atomicOr(&p.st->err, NB_DEV_CLUSTER_OVERFLOW);
            nout = NB_CI_ENTRY_BUF;
        }
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&p.st->list_count, (unsigned long long)nout);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base + (unsigned long long)nout > p.cap) {
            if (lane == 0) atomicOr(&p.st->err, NB_DEV_LIST_OVERFLOW);
            nout = 0;
            base = 0;
        }
        for (int k = lane; k < nout; k += 32) p.outer[base + k] = buf[k];
        if (lane == 0) {
            p.ci_start[ci] = (int)base;
            p.ci_len[ci] = nout;
            p.ci_len_inner[ci] = 0;
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t nb_launch_search(nb_pairlist *pl, const int *excl_off, const int *excl_idx, float rl2,
                             float rl_col, cudaStream_t s) {
    SearchParams p;
    p.bbox = pl->bbox;
    p.col_clus_start = pl->col_clus_start;
    p.perm = pl->perm;
    p.pos = pl->pos;
    p.excl_off = excl_off;
    p.excl_idx = excl_idx;
    p.outer = pl->outer;
    p.ci_start = pl->ci_start;
    p.ci_len = pl->ci_len_outer;
    p.ci_len_inner = pl->ci_len_inner;
    p.st = pl->st;
    p.sys = pl->sys;
    p.clus_sys = pl->clus_sys;
    p.n_atoms = pl->n_atoms;
    p.rl2 = rl2;
    p.rl_col = rl_col;
    p.cap = (unsigned long long)pl->cap;
    const size_t smem = sizeof(int4) * kSearchWarps * NB_CI_ENTRY_BUF;
    // once per device (outside any stream capture: the first search on a
    // device must not be captured)
    static bool attr_done[64] = {};
    if (pl->device < 0 || pl->device >= 64 || !attr_done[pl->device]) {
        cudaError_t e = cudaFuncSetAttribute(k_search, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (pl->device >= 0 && pl->device < 64) attr_done[pl->device] = true;
    }
    int blocks = (pl->nc_max + kSearchWarps - 1) / kSearchWarps;
    blocks = min(blocks, pl->num_sms * 16);
    k_search<<<blocks, kSearchWarps * 32, smem, s>>>(p);
    return cudaGetLastError();
}
