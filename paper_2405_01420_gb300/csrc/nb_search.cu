// Cluster-pair search: the outer ("buffered") pair list at radius rlist
// (§III-A: "pair list buffer", "list range").
//
// One warp per i-cluster ci. The warp walks the grid columns whose xy extent
// lies within rlist of ci's bounding box (with periodic images), and in each
// column tests the clusters cj >= ci, one per lane, by bounding-box distance.
// Kept pairs get a shift index and a 64-bit mask (bit a*8+b: atom a of ci
// with atom b of cj) of real, non-excluded, non-duplicated atom pairs. The
// warp stages the kept pairs, reserves space in the list with one atomic,
// and writes them out, coalesced.
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
    const int *ztab;  // per column: first cluster whose upper z bound reaches k Lz / NB_ZBINS
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

constexpr int kExclTab = 64;  // clusters holding excluded partners of one i-cluster
constexpr int kSearchBuf = 128;  // kept pairs of one i-cluster staged in shared memory

// Per-warp shared state of the candidate walk.
struct WalkShared {
    int incl[32];     // inclusive prefix of the candidates of the batch's columns
    int cs[3][32];    // first candidate cluster of each z image of each column
    int len01[32];    // candidates of the column's first two z images (16 bits each)
    int zpack[32];    // kz + 1 of the column's z images, 2 bits each (up to 3); kx + 1 at bit 8, ky + 1 at bit 10
};

// First cluster c in [a, b) with bbox[2c + hi].z >= z (hi = 1) or > z
// (hi = 0, strict), for z-sorted clusters of one column: their lower and
// upper z bounds are both non-decreasing in c (the column's atoms are
// sorted by z and a cluster holds consecutive ones). zt is the column's z
// index: every cluster before zt[k] has its upper bound below k dz, so for
// k dz <= z neither test can hold there; k one bin below z's keeps the
// start clear of rounding, and a short forward scan finds the answer.
__device__ __forceinline__ int z_first(const float4 *bbox, const int *zt, int a, int b, int hi, float z,
                                       float inv_dz) {
    const int k = min(max((int)floorf(z * inv_dz) - 1, 0), NB_ZBINS);
    int c = max(a, zt[k]);
    while (c < b) {
        const float v = bbox[2 * c + hi].z;
        if (hi ? v >= z : v > z) break;
        ++c;
    }
    return c;
}

// Walks the candidate clusters of ci: the grid columns within rl_col of its
// bounding box (with periodic images), their z images, and in each the
// clusters cj >= ci whose z extent comes within rl_col of ci's (found from
// the column's z index; a column spans the whole box in z). A
// batch of 32 columns is read in parallel (one per lane); a warp scan lays
// their candidates end to end, and the lanes then test 32 candidates at a
// time (the column of a candidate found by binary search over the scan). visit(c, sidx, m, r) is called by every lane that
// keeps its pair (bounding boxes within rl2 and a non-empty mask m of real,
// non-excluded, non-duplicated atom pairs), with its rank r among the kept
// ones; the order is fixed, so two walks make the same calls.
template <typename Visit>
__device__ __forceinline__ int walk_candidates(const SearchParams &p, int ci, const float4 lo, const float4 hi, int ni,
                                               const nb_sys &S, const int *tab_c, const unsigned long long *tab_m,
                                               int ntab, int tlo, int thi, WalkShared &ws, int lane, Visit visit) {
    int nout = 0;
    const int jx0 = max((int)floorf((lo.x - p.rl_col) * S.inv_sx), -S.ncx);
    const int jx1 = min((int)floorf((hi.x + p.rl_col) * S.inv_sx), 2 * S.ncx - 1);
    const int jy0 = max((int)floorf((lo.y - p.rl_col) * S.inv_sy), -S.ncy);
    const int jy1 = min((int)floorf((hi.y + p.rl_col) * S.inv_sy), 2 * S.ncy - 1);
    const int nyr = jy1 - jy0 + 1;
    const int ncols = (jx1 - jx0 + 1) * nyr;
    const float inv_nyr = 1.0f / (float)nyr;
    // cell edges; the binning's boundaries differ from these products by rounding only, far
    // below the 1e-3 nm by which rl_col exceeds the list radius
    const float csx = S.box.x / (float)S.ncx, csy = S.box.y / (float)S.ncy;
    const float inv_dz = (float)NB_ZBINS / S.box.z;
    const float rl_col2 = p.rl_col * p.rl_col;
    for (int kb = 0; kb < ncols; kb += 32) {
        // this lane's column: its candidate range and z images
        const int k = kb + lane;
        int cs0 = 0, cs1 = 0, cs2 = 0, len0 = 0, len1 = 0, len2 = 0;
        int zpack = 0, nz = 0;
        if (k < ncols) {
            // k = kxr * nyr + kyr; the float quotient is off by at most one for these small integers
            int kxr = (int)((float)k * inv_nyr);
            kxr += (kxr + 1) * nyr <= k;
            kxr -= kxr * nyr > k;
            const int jxu = jx0 + kxr, jyu = jy0 + (k - kxr * nyr);
            const int kx = image_of(jxu, S.ncx), ky = image_of(jyu, S.ncy);
            const int jx = jxu - kx * S.ncx, jy = jyu - ky * S.ncy;
            const int col = S.col_off + jx * S.ncy + jy;
            // the column's cell (this image) in the xy plane; a cell farther than rl_col from ci's box
            // (a corner of the square of columns) holds no candidate
            const float cx0 = (float)jxu * csx, cy0 = (float)jyu * csy;
            const float gx = fmaxf(0.0f, fmaxf(cx0 - hi.x, lo.x - (cx0 + csx)));
            const float gy = fmaxf(0.0f, fmaxf(cy0 - hi.y, lo.y - (cy0 + csy)));
            const bool near = gx * gx + gy * gy < rl_col2;
            const int c0 = max(p.col_clus_start[col], ci), c1 = near ? p.col_clus_start[col + 1] : 0;
            const int *zt = p.ztab + col * (NB_ZBINS + 1);
            zpack = ((kx + 1) << 8) | ((ky + 1) << 10);
            for (int kz = -1; kz <= 1 && c0 < c1; ++kz) {
                // clusters whose z extent, moved by oz, comes within rl_col of ci's
                const float oz = (float)kz * S.box.z;
                const float zlo = (lo.z - p.rl_col) - oz, zhi = (hi.z + p.rl_col) - oz;
                const int a = z_first(p.bbox, zt, c0, c1, 1, zlo, inv_dz);
                const int b = z_first(p.bbox, zt, a, c1, 0, zhi, inv_dz);
                if (b <= a) continue;
                if (nz == 0) {
                    cs0 = a;
                    len0 = b - a;
                } else if (nz == 1) {
                    cs1 = a;
                    len1 = b - a;
                } else {
                    cs2 = a;
                    len2 = b - a;
                }
                zpack |= (kz + 1) << (2 * nz);
                ++nz;
            }
        }
        const int tot = len0 + len1 + len2;
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
        ws.incl[lane] = incl;
        ws.cs[0][lane] = cs0;
        ws.cs[1][lane] = cs1;
        ws.cs[2][lane] = cs2;
        ws.len01[lane] = len0 | (len1 << 16);  // a column holds at most NB_MAX_COL_ATOMS / 8 clusters
        ws.zpack[lane] = zpack;
        __syncwarp();
        for (int u0 = 0; u0 < total; u0 += 32) {
            const int u = u0 + lane;
            bool keep = false;
            unsigned long long m = 0;
            int c = 0, sidx = 0;
            if (u < total) {
                int o = 0;  // the column holding candidate u: columns with incl <= u come first
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1)
                    if (ws.incl[o + step - 1] <= u) o += step;
                const int lp = ws.len01[o];
                const int l0 = lp & 0xffff, l01 = l0 + (lp >> 16);
                const int first = (o == 0 ? 0 : ws.incl[o - 1]);
                const int w = u - first;                 // index within the column's candidates
                const int zi = (w >= l0) + (w >= l01);   // which z image (at most 3)
                const int zp = ws.zpack[o];
                const int kz = ((zp >> (2 * zi)) & 3) - 1;
                c = ws.cs[zi][o] + (w - (zi == 0 ? 0 : (zi == 1 ? l0 : l01)));
                const int kx = ((zp >> 8) & 3) - 1, ky = ((zp >> 10) & 3) - 1;
                sidx = (1 - kx) * 9 + (1 - ky) * 3 + 1 - kz;
                // j image at x_b + ox, i.e. S_x = -ox
                const float oxo = (float)kx * S.box.x, oyo = (float)ky * S.box.y;
                const float oz = (float)kz * S.box.z;
                const float4 bl = p.bbox[2 * c], bh = p.bbox[2 * c + 1];
                const float gx = fmaxf(0.0f, fmaxf((bl.x + oxo) - hi.x, lo.x - (bh.x + oxo)));
                const float gy = fmaxf(0.0f, fmaxf((bl.y + oyo) - hi.y, lo.y - (bh.y + oyo)));
                const float gz = fmaxf(0.0f, fmaxf((bl.z + oz) - hi.z, lo.z - (bh.z + oz)));
                keep = gx * gx + gy * gy + gz * gz < p.rl2;
                if (c == ci && sidx < NB_SHIFT_CENTER) keep = false;
                if (keep) {
                    const int nj = __float_as_int(bl.w);
                    m = row_mask(ni) * (unsigned long long)((1u << nj) - 1u);
                    if (c == ci) m &= (sidx == NB_SHIFT_CENTER) ? kUpperStrict : ~kDiagonal;
                    if (c >= tlo && c <= thi)
                        for (int q = 0; q < ntab; ++q)
                            if (tab_c[q] == c) m &= ~tab_m[q];
                    keep = (m != 0ull);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) visit(c, sidx, m, nout + __popc(bal & ((1u << lane) - 1u)));
            nout += __popc(bal);
        }
    }
    return nout;
}

// One warp per i-cluster. The exclusions of ci's atoms are folded into a
// table of (j cluster, 64-bit mask of excluded pairs). The walk stages the
// kept pairs in shared memory, one atomic reserves exactly that many list
// entries, and the warp copies them out coalesced; a list longer than the
// stage is written by a second walk (the same decisions) instead.
__global__ void __launch_bounds__(kSearchWarps * 32, 4) k_search(SearchParams p) {
    __shared__ int2 s_excl[kSearchWarps][NB_CI_EXCL_BUF];
    __shared__ int s_nexcl[kSearchWarps];
    __shared__ int s_tab_c[kSearchWarps][kExclTab];
    __shared__ unsigned long long s_tab_m[kSearchWarps][kExclTab];
    __shared__ WalkShared s_walk[kSearchWarps];
    __shared__ int4 s_buf[kSearchWarps][kSearchBuf];
    nb_pdl_wait();  // with programmatic dependent launch: the grid sort has completed from here on
    nb_pdl_release();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
        // fold them by j cluster (a handful of clusters per i-cluster), warp-wide: in each round of
        // 32 entries the lanes of one j cluster elect their lowest lane, which ORs their bits and
        // files them (in a new table entry, or in the entry of an earlier round)
        int ntab = 0;
        for (int r0 = 0; r0 < nex; r0 += 32) {
            const int e = r0 + lane;
            const bool valid = e < nex;
            const int cj = valid ? (s_excl[warp][e].y >> 3) : -1 - lane;  // idle lanes match nobody
            const unsigned peers = __match_any_sync(0xffffffffu, cj);
            const bool lead = valid && __ffs(peers) - 1 == lane;
            unsigned long long m = 0ull;
            int k = -1;
            if (lead) {
                for (unsigned q = peers; q; q &= q - 1u) {
                    const int2 ex = s_excl[warp][r0 + __ffs(q) - 1];
                    m |= 1ull << (ex.x * 8 + (ex.y & 7));
                }
                for (int t = 0; t < ntab; ++t)
                    if (s_tab_c[warp][t] == cj) {
                        k = t;
                        break;
                    }
            }
            const bool fresh = lead && k < 0;
            const unsigned fr = __ballot_sync(0xffffffffu, fresh);
            if (fresh) k = ntab + __popc(fr & ((1u << lane) - 1u));
            if (lead) {
                if (k >= kExclTab) {
                    atomicOr(&p.st->err, NB_DEV_EXCL_OVERFLOW);
                } else if (fresh) {
                    s_tab_c[warp][k] = cj;
                    s_tab_m[warp][k] = m;
                } else {
                    s_tab_m[warp][k] |= m;
                }
            }
            ntab = min(ntab + __popc(fr), kExclTab);
            __syncwarp();
        }
        // the range of the table's clusters: most candidates fall outside it
        int tlo = 0x7fffffff, thi = -1;
        for (int t = lane; t < ntab; t += 32) {
            tlo = min(tlo, s_tab_c[warp][t]);
            thi = max(thi, s_tab_c[warp][t]);
        }
        tlo = __reduce_min_sync(0xffffffffu, tlo);
        thi = __reduce_max_sync(0xffffffffu, thi);
        const int *tab_c = s_tab_c[warp];
        const unsigned long long *tab_m = s_tab_m[warp];

        // first walk: kept pairs into the warp's buffer (while they fit)
        int4 *buf = s_buf[warp];
        const int nout = walk_candidates(p, ci, lo, hi, ni, S, tab_c, tab_m, ntab, tlo, thi, s_walk[warp], lane,
                                         [buf](int c, int sidx, unsigned long long m, int r) {
                                             if (r < kSearchBuf)
                                                 buf[r] = make_int4(c, sidx, (int)(unsigned)(m & 0xffffffffu),
                                                                    (int)(unsigned)(m >> 32));
                                         });
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&p.st->list_count, (unsigned long long)nout);
        base = __shfl_sync(0xffffffffu, base, 0);
        int nkept = nout;
        __syncwarp();
        if (base + (unsigned long long)nout > p.cap) {
            if (lane == 0) atomicOr(&p.st->err, NB_DEV_LIST_OVERFLOW);
            nkept = 0;
            base = 0;
        } else if (nout <= kSearchBuf) {
            for (int k = lane; k < nout; k += 32) p.outer[base + k] = buf[k];
        } else {  // a long list: a second walk writes it directly
            int4 *out = p.outer + base;
            walk_candidates(p, ci, lo, hi, ni, S, tab_c, tab_m, ntab, tlo, thi, s_walk[warp], lane,
                            [out](int c, int sidx, unsigned long long m, int r) {
                                out[r] = make_int4(c, sidx, (int)(unsigned)(m & 0xffffffffu), (int)(unsigned)(m >> 32));
                            });
        }
        if (lane == 0) {
            p.ci_start[ci] = (int)base;
            p.ci_len[ci] = nkept;
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
    p.ztab = pl->ztab;
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
    int blocks = (pl->nc_max + kSearchWarps - 1) / kSearchWarps;
    blocks = min(blocks, pl->num_sms * 16);
    return nb_launch_if(pl->nc_max <= NB_SEARCH_PDL_MAX_CLUSTERS, k_search, blocks, kSearchWarps * 32, 0, s, p);
}
