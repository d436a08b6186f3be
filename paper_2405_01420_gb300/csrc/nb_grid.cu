// Grid sort into 8-atom clusters (first stage of the pair search, §III-A).
//
// 0. k_search_begin: clear the column counts and the list counter; write a
//    single system's table.
// 1. k_bin: wrap each atom into the box and bin it into an xy column;
//    count atoms per column.
// 2. k_col_scan: exclusive scans of atoms and of 8-atom clusters per column.
// 3. k_col_scatter: bucket (z, atom) keys by column.
// 4. k_col_sort: sorts each column's keys by z (bitonic: in one warp's
//    registers up to 256 atoms, else by a CTA in shared memory), packs runs
//    of 8 into clusters, pads the last one, and writes the slot <-> atom
//    maps, the search-frame positions and per-cluster bounding boxes.
//
// Layout in HBM after the sort (slot = 8 * cluster + lane):
//   perm[slot] (int), xref[slot] (float4), bbox[2c], bbox[2c+1] (float4).
#include <algorithm>
#include <cstring>

#include "nb_internal.cuh"

namespace {

// The start of a search: clears the column counts and the list counter and,
// for a single-system pair list, writes its system table (one entry and its
// 27 shift vectors) from kernel arguments, so that a search can be captured
// in a CUDA graph without a host-to-device copy. Like every kernel of the
// grid sort and the search it may be launched with programmatic dependent
// launch (nb_launch_if, for lists up to NB_SEARCH_PDL_MAX_CLUSTERS).
__global__ void k_search_begin(nb_sys *sys, float4 *sys_shift, nb_sys one, int write_sys, int *col_count, int ncol,
                               nb_dev_state *st) {
    nb_pdl_wait();
    nb_pdl_release();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncol; k += gridDim.x * blockDim.x) col_count[k] = 0;
    if (blockIdx.x != 0) return;
    const int k = threadIdx.x;
    if (k == 0) st->list_count = 0ull;
    if (!write_sys) return;
    if (k == 0) sys[0] = one;
    if (k < 27)
        sys_shift[k] = make_float4((float)nb_shift_x(k) * one.box.x, (float)nb_shift_y(k) * one.box.y,
                                   (float)nb_shift_z(k) * one.box.z, 0.0f);
}

__global__ void k_bin(int n, const float *__restrict__ coords, const int *__restrict__ atom_sys,
                      const nb_sys *__restrict__ sys, int *__restrict__ col_count, int *__restrict__ atom_col,
                      int *__restrict__ atom_slot, float4 *__restrict__ xw, nb_dev_state *st) {
    nb_pdl_wait();
    nb_pdl_release();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int col = -1 - lane;  // lanes past the end match nobody below
    if (i < n) {
        const nb_sys S = sys[atom_sys[i]];
        float x = coords[3 * i + 0], y = coords[3 * i + 1], z = coords[3 * i + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
            atomicOr(&st->err, NB_DEV_NONFINITE);
            x = 0.0f;
            y = 0.0f;
            z = 0.0f;
        }
        float4 w = make_float4(nb_wrap(x, S.box.x), nb_wrap(y, S.box.y), nb_wrap(z, S.box.z), 0.0f);
        int cx = min(S.ncx - 1, max(0, (int)floorf(w.x * S.inv_sx)));
        int cy = min(S.ncy - 1, max(0, (int)floorf(w.y * S.inv_sy)));
        col = S.col_off + cx * S.ncy + cy;
        xw[i] = w;
        atom_col[i] = col;
    }
    // arrival ranks within the column: one atomic per group of lanes in the same column (neighbouring
    // atoms often share one, and atomics on one counter serialise); the per-column sort orders the
    // atoms by (z, index) afterwards, so the ranks' order does not show in the result
    const unsigned peers = __match_any_sync(0xffffffffu, col);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (i < n && lane == leader) base = atomicAdd(&col_count[col], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (i < n) atom_slot[i] = base + __popc(peers & ((1u << lane) - 1u));
}

// Single CTA: exclusive scans of col_count (atoms) and ceil(count/8)
// (clusters) over ncol columns; total clusters -> st->nc.
__global__ void __launch_bounds__(1024) k_col_scan(int ncol, const int *__restrict__ col_count,
                                                   int *__restrict__ col_atom_start,
                                                   int *__restrict__ col_clus_start,
                                                   nb_dev_state *st) {
    nb_pdl_wait();
    nb_pdl_release();
    __shared__ int warp_a[32], warp_c[32];
    int t = threadIdx.x, nt = blockDim.x;
    int chunk = (ncol + nt - 1) / nt;
    int b = t * chunk, e = min(ncol, b + chunk);
    int sa = 0, sc = 0, over = 0;
    // Atom offsets use the full counts (every atom gets a key slot); cluster
    // offsets use the counts the per-column sort can hold, so that every
    // allocated cluster slot is written even after a column overflow.
    for (int c = b; c < e; ++c) {
        int k = col_count[c];
        sa += k;
        sc += (min(k, NB_MAX_COL_ATOMS) + NB_CLUSTER - 1) / NB_CLUSTER;
        over |= (k > NB_MAX_COL_ATOMS);
    }
    if (over) atomicOr(&st->err, NB_DEV_COLUMN_OVERFLOW);
    // inclusive scan of (sa, sc) across the CTA
    int lane = t & 31, wid = t >> 5;
    int ia = sa, ic = sc;
    for (int o = 1; o < 32; o <<= 1) {
        int va = __shfl_up_sync(0xffffffffu, ia, o), vc = __shfl_up_sync(0xffffffffu, ic, o);
        if (lane >= o) {
            ia += va;
            ic += vc;
        }
    }
    if (lane == 31) {
        warp_a[wid] = ia;
        warp_c[wid] = ic;
    }
    __syncthreads();
    if (wid == 0) {
        int nw = nt >> 5;
        int va = lane < nw ? warp_a[lane] : 0, vc = lane < nw ? warp_c[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int ua = __shfl_up_sync(0xffffffffu, va, o), uc = __shfl_up_sync(0xffffffffu, vc, o);
            if (lane >= o) {
                va += ua;
                vc += uc;
            }
        }
        warp_a[lane] = va;
        warp_c[lane] = vc;
    }
    __syncthreads();
    int pa = (wid > 0 ? warp_a[wid - 1] : 0) + ia - sa;  // exclusive prefix of this thread
    int pc = (wid > 0 ? warp_c[wid - 1] : 0) + ic - sc;
    for (int c = b; c < e; ++c) {
        col_atom_start[c] = pa;
        col_clus_start[c] = pc;
        int k = col_count[c];
        pa += k;
        pc += (min(k, NB_MAX_COL_ATOMS) + NB_CLUSTER - 1) / NB_CLUSTER;
    }
    if (t == nt - 1) {
        col_atom_start[ncol] = pa;
        col_clus_start[ncol] = pc;
        st->nc = pc;
    }
}

__global__ void k_col_scatter(int n, const float4 *__restrict__ xw, const int *__restrict__ atom_col,
                              const int *__restrict__ atom_slot,
                              const int *__restrict__ col_atom_start,
                              unsigned long long *__restrict__ keys) {
    nb_pdl_wait();
    nb_pdl_release();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // z >= 0 after wrapping, so its bit pattern orders like the value
    unsigned long long k = ((unsigned long long)__float_as_uint(xw[i].z) << 32) | (unsigned)i;
    keys[col_atom_start[atom_col[i]] + atom_slot[i]] = k;
}

struct ColSortParams {
    const int *col_count;
    const int *col_atom_start;
    const int *col_clus_start;
    const unsigned long long *keys;
    const float4 *xw;
    const int *col_sys;
    int *perm;
    int *pos;
    float4 *xref;
    float4 *xprune;
    float4 *xq;
    int *tsort;
    float4 *bbox;
    int *clus_sys;
    const nb_sys *sys;
    int *ztab;
    int ncol;
    int cpc;  // columns per CTA, 1 .. kSortWarps: warp w < cpc takes column cpc * blockIdx.x + w
};

constexpr int kSortWarps = 8;       // columns per CTA, one per warp
constexpr int kWarpSortKeys = 256;  // a column up to this size is sorted in one warp's registers

// Compare-exchange: a <= b afterwards if up, a >= b otherwise.
__device__ __forceinline__ void cmpx(unsigned long long &a, unsigned long long &b, bool up) {
    const bool swap = (a > b) == up;
    const unsigned long long t = a;
    a = swap ? b : a;
    b = swap ? t : b;
}

// Bitonic sort, ascending, of the 256 keys of a warp: key 8 lane + j in v[j].
// Strides below 8 pair two registers of one lane; a stride s >= 8 pairs lane
// l with lane l ^ (s / 8), and each of the two keeps the lower or the higher
// of its exchanged keys.
__device__ __forceinline__ void warp_bitonic_sort(unsigned long long (&v)[8], int lane) {
#pragma unroll
    for (int size = 2; size <= kWarpSortKeys; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 8) {
                const int lm = stride >> 3;
                const bool up = ((8 * lane) & size) == 0;
                const bool keep_lo = up == ((lane & lm) == 0);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[j], lm);
                    v[j] = keep_lo ? (o < v[j] ? o : v[j]) : (o > v[j] ? o : v[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if ((j ^ stride) > j) cmpx(v[j], v[j ^ stride], ((8 * lane + j) & size) == 0);
            }
        }
    }
}

// The rest of a column once its cnt keys are sorted by z in sk: its z index,
// its slot <-> atom maps, search-frame positions and padding, and its
// clusters' bounding boxes. G threads (t = 0 .. G - 1) take part, G a
// multiple of 32: the 8 slots of a cluster are 8 aligned lanes of a warp,
// which reduce the bounding box over its real atoms with shuffles.
template <int G>
__device__ __forceinline__ void finish_column(const ColSortParams &p, const unsigned long long *sk, int cnt,
                                              int col, int t) {
    const int c0 = p.col_clus_start[col];
    const int ncl = (cnt + NB_CLUSTER - 1) / NB_CLUSTER;
    const int s0 = c0 * NB_CLUSTER;
    const float4 pad = make_float4(NB_PAD_COORD, NB_PAD_COORD, NB_PAD_COORD, 0.0f);
    const int csys = p.col_sys[col];
    // the column's z index: per bin k, the first cluster whose upper z bound (its last atom's z; the
    // keys are sorted by z) reaches k Lz / NB_ZBINS
    for (int zb_k = t; zb_k <= NB_ZBINS; zb_k += G) {
        const float zb = (float)zb_k * (p.sys[csys].box.z / (float)NB_ZBINS);
        int a = 0, b = ncl;
        while (a < b) {
            const int m = (a + b) >> 1;
            const float hz = __uint_as_float((unsigned)(sk[min(NB_CLUSTER * m + NB_CLUSTER - 1, cnt - 1)] >> 32));
            if (hz >= zb)
                b = m;
            else
                a = m + 1;
        }
        p.ztab[col * (NB_ZBINS + 1) + zb_k] = c0 + a;
    }
    const int nslots = ncl * NB_CLUSTER;
    for (int k0 = 0; k0 < nslots; k0 += G) {
        const int k = k0 + t;
        const int slot = s0 + k;
        float4 lo = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.0f), hi = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.0f);
        if (k < cnt) {
            const int atom = (int)(sk[k] & 0xffffffffu);
            const float4 w = p.xw[atom];
            p.perm[slot] = atom;
            p.pos[atom] = slot;
            p.xref[slot] = w;
            p.xprune[slot] = w;
            lo = make_float4(w.x, w.y, w.z, 0.0f);
            hi = lo;
        } else if (k < nslots) {
            p.perm[slot] = -1;
            p.xref[slot] = pad;
            p.xprune[slot] = pad;
            p.xq[slot] = pad;
            p.tsort[slot] = 0;
        }
#pragma unroll
        for (int o = 1; o < NB_CLUSTER; o <<= 1) {
            lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
            lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
            lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
            hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
            hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
            hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
        }
        if (k < nslots && (k & (NB_CLUSTER - 1)) == 0) {
            const int c = k / NB_CLUSTER;
            const int nreal = min(NB_CLUSTER, cnt - k);
            lo.w = __int_as_float(nreal);
            hi.w = __int_as_float(col);
            p.bbox[2 * (c0 + c)] = lo;
            p.bbox[2 * (c0 + c) + 1] = hi;
            p.clus_sys[c0 + c] = csys;
        }
    }
}

// cpc columns per CTA. With several (short columns on average), a column of
// at most kWarpSortKeys atoms is sorted by one warp in registers (no block
// barriers) and a longer one, after those, by the whole CTA with a bitonic
// sort in shared memory. The launch takes one column per CTA when columns
// hold more than kWarpSortKeys / 2 atoms on average; the whole CTA then
// sorts it (one warp alone was slower: its 36 dependent shuffle stages are
// not shared out). Shared memory: NB_MAX_COL_ATOMS keys, kWarpSortKeys of
// them per warp for short columns.
__global__ void __launch_bounds__(kSortWarps * 32) k_col_sort(ColSortParams p) {
    static_assert(kSortWarps * kWarpSortKeys <= NB_MAX_COL_ATOMS, "warp regions exceed the key buffer");
    __shared__ unsigned long long sk[NB_MAX_COL_ATOMS];
    nb_pdl_wait();
    nb_pdl_release();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col0 = blockIdx.x * p.cpc;
    const int warp_max = p.cpc > 1 ? kWarpSortKeys : 0;  // the longest column a warp sorts alone
    if (warp < p.cpc) {
        const int col = col0 + warp;
        const int cnt = col < p.ncol ? min(p.col_count[col], NB_MAX_COL_ATOMS) : 0;
        if (col < p.ncol && cnt <= warp_max) {
            const int a0 = p.col_atom_start[col];
            unsigned long long v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = 8 * lane + j;
                v[j] = k < cnt ? p.keys[a0 + k] : ~0ull;
            }
            warp_bitonic_sort(v, lane);
            unsigned long long *sw = sk + warp * kWarpSortKeys;
#pragma unroll
            for (int j = 0; j < 8; ++j) sw[8 * lane + j] = v[j];
            __syncwarp();
            finish_column<32>(p, sw, cnt, col, lane);
        }
    }
    for (int w = 0; w < p.cpc; ++w) {  // the same decisions in every thread of the CTA
        const int col = col0 + w;
        if (col >= p.ncol) break;
        const int cnt = min(p.col_count[col], NB_MAX_COL_ATOMS);  // overflow already flagged by the scan
        if (cnt <= warp_max) continue;
        __syncthreads();  // every earlier use of sk is over
        const int a0 = p.col_atom_start[col];
        int p2 = 1;
        while (p2 < cnt) p2 <<= 1;
        for (int k = threadIdx.x; k < p2; k += blockDim.x) sk[k] = (k < cnt) ? p.keys[a0 + k] : ~0ull;
        __syncthreads();
        for (int size = 2; size <= p2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int k = threadIdx.x; k < p2; k += blockDim.x) {
                    const int partner = k ^ stride;
                    if (partner > k) {
                        const bool up = ((k & size) == 0);
                        const unsigned long long u = sk[k], v = sk[partner];
                        if ((u > v) == up) {
                            sk[k] = v;
                            sk[partner] = u;
                        }
                    }
                }
                __syncthreads();
            }
        }
        finish_column<kSortWarps * 32>(p, sk, cnt, col, threadIdx.x);
    }
}

}  // namespace

cudaError_t nb_launch_grid_sort(nb_pairlist *pl, const float *coords, const nb_sys *one, cudaStream_t s) {
    const int n = pl->n_atoms;
    const bool pdl = pl->nc_max <= NB_SEARCH_PDL_MAX_CLUSTERS;
    nb_sys none;
    std::memset(&none, 0, sizeof(none));
    const int bs = 256, gb = (n + bs - 1) / bs;
    const int gc = std::max(1, std::min((pl->ncol + bs - 1) / bs, 4 * pl->num_sms));
    cudaError_t e = nb_launch_if(pdl, k_search_begin, gc, bs, 0, s, pl->sys, pl->sys_shift, one ? *one : none,
                                  one ? 1 : 0, pl->col_count, pl->ncol, pl->st);
    if (e != cudaSuccess) return e;
    e = nb_launch_if(pdl, k_bin, gb, bs, 0, s, n, coords, (const int *)pl->atom_sys, (const nb_sys *)pl->sys,
                      pl->col_count, pl->atom_col, pl->atom_slot, pl->xw, pl->st);
    if (e != cudaSuccess) return e;
    e = nb_launch_if(pdl, k_col_scan, 1, 1024, 0, s, pl->ncol, (const int *)pl->col_count, pl->col_atom_start,
                      pl->col_clus_start, pl->st);
    if (e != cudaSuccess) return e;
    e = nb_launch_if(pdl, k_col_scatter, gb, bs, 0, s, n, (const float4 *)pl->xw, (const int *)pl->atom_col,
                      (const int *)pl->atom_slot, (const int *)pl->col_atom_start, pl->keys);
    if (e != cudaSuccess) return e;
    ColSortParams cp;
    cp.col_count = pl->col_count;
    cp.col_atom_start = pl->col_atom_start;
    cp.col_clus_start = pl->col_clus_start;
    cp.keys = pl->keys;
    cp.xw = pl->xw;
    cp.col_sys = pl->col_sys;
    cp.perm = pl->perm;
    cp.pos = pl->pos;
    cp.xref = pl->xref;
    cp.xprune = pl->xprune;
    cp.xq = pl->xq;
    cp.tsort = pl->tsort;
    cp.bbox = pl->bbox;
    cp.clus_sys = pl->clus_sys;
    cp.sys = pl->sys;
    cp.ztab = pl->ztab;
    cp.ncol = pl->ncol;
    cp.cpc = (long long)n <= (long long)pl->ncol * (kWarpSortKeys / 2) ? kSortWarps : 1;
    return nb_launch_if(pdl, k_col_sort, (pl->ncol + cp.cpc - 1) / cp.cpc, kSortWarps * 32, 0, s, cp);
}
