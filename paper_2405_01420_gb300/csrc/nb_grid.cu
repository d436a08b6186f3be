// Grid sort into 8-atom clusters (first stage of the pair search, §III-A).
//
// 1. k_bin: wrap each atom into the box and bin it into an xy column;
//    count atoms per column.
// 2. k_col_scan: exclusive scans of atoms and of 8-atom clusters per column.
// 3. k_col_scatter: bucket (z, atom) keys by column.
// 4. k_col_sort: one CTA per column sorts its keys by z (bitonic, shared
//    memory), packs runs of 8 into clusters, pads the last one, and writes
//    the slot <-> atom maps, the search-frame positions and per-cluster
//    bounding boxes.
//
// Layout in HBM after the sort (slot = 8 * cluster + lane):
//   perm[slot] (int), xref[slot] (float4), bbox[2c], bbox[2c+1] (float4).
#include "nb_internal.cuh"

namespace {

// Writes the system table of a single-system pair list (one entry and its
// 27 shift vectors) from kernel arguments, so that a search can be captured
// in a CUDA graph without a host-to-device copy.
__global__ void k_set_system(nb_sys *sys, float4 *sys_shift, nb_sys one) {
    const int k = threadIdx.x;
    if (k == 0) sys[0] = one;
    if (k < 27)
        sys_shift[k] = make_float4((float)nb_shift_x(k) * one.box.x, (float)nb_shift_y(k) * one.box.y,
                                   (float)nb_shift_z(k) * one.box.z, 0.0f);
}

__global__ void k_bin(int n, const float *__restrict__ coords, const int *__restrict__ atom_sys,
                      const nb_sys *__restrict__ sys, int *__restrict__ col_count, int *__restrict__ atom_col,
                      int *__restrict__ atom_slot, float4 *__restrict__ xw, nb_dev_state *st) {
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
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // z >= 0 after wrapping, so its bit pattern orders like the value
    unsigned long long k = ((unsigned long long)__float_as_uint(xw[i].z) << 32) | (unsigned)i;
    keys[col_atom_start[atom_col[i]] + atom_slot[i]] = k;
}

// One CTA per column. Shared memory: NB_MAX_COL_ATOMS keys.
__global__ void __launch_bounds__(256) k_col_sort(
    const int *__restrict__ col_count, const int *__restrict__ col_atom_start,
    const int *__restrict__ col_clus_start, const unsigned long long *__restrict__ keys,
    const float4 *__restrict__ xw, const int *__restrict__ col_sys, int *__restrict__ perm,
    int *__restrict__ pos, float4 *__restrict__ xref, float4 *__restrict__ xprune, float4 *__restrict__ xq,
    int *__restrict__ tsort, float4 *__restrict__ bbox, int *__restrict__ clus_sys, const nb_sys *__restrict__ sys,
    int *__restrict__ ztab) {
    __shared__ unsigned long long sk[NB_MAX_COL_ATOMS];
    int col = blockIdx.x;
    int cnt = min(col_count[col], NB_MAX_COL_ATOMS);  // overflow already flagged by the scan
    int a0 = col_atom_start[col];
    int p2 = 1;
    while (p2 < cnt) p2 <<= 1;
    for (int k = threadIdx.x; k < p2; k += blockDim.x) sk[k] = (k < cnt) ? keys[a0 + k] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= p2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < p2; k += blockDim.x) {
                int partner = k ^ stride;
                if (partner > k) {
                    bool up = ((k & size) == 0);
                    unsigned long long u = sk[k], v = sk[partner];
                    if ((u > v) == up) {
                        sk[k] = v;
                        sk[partner] = u;
                    }
                }
            }
            __syncthreads();
        }
    }
    int c0 = col_clus_start[col];
    int ncl = (cnt + NB_CLUSTER - 1) / NB_CLUSTER;
    int s0 = c0 * NB_CLUSTER;
    const float4 pad = make_float4(NB_PAD_COORD, NB_PAD_COORD, NB_PAD_COORD, 0.0f);
    const int csys = col_sys[col];
    // the column's z index: per bin k, the first cluster whose upper z bound (its last atom's z; the
    // keys are sorted by z) reaches k Lz / NB_ZBINS
    if (threadIdx.x <= NB_ZBINS) {
        const float zb = (float)threadIdx.x * (sys[csys].box.z / (float)NB_ZBINS);
        int a = 0, b = ncl;
        while (a < b) {
            const int m = (a + b) >> 1;
            const float hz = __uint_as_float((unsigned)(sk[min(NB_CLUSTER * m + NB_CLUSTER - 1, cnt - 1)] >> 32));
            if (hz >= zb)
                b = m;
            else
                a = m + 1;
        }
        ztab[col * (NB_ZBINS + 1) + threadIdx.x] = c0 + a;
    }
    // one thread per slot; the 8 slots of a cluster are 8 aligned lanes of a warp, which reduce the
    // cluster's bounding box over its real atoms with shuffles (every lane of a warp takes part)
    const int nslots = ncl * NB_CLUSTER;
    for (int k0 = 0; k0 < nslots; k0 += blockDim.x) {
        const int k = k0 + (int)threadIdx.x;
        const int slot = s0 + k;
        float4 lo = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.0f), hi = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.0f);
        if (k < cnt) {
            int atom = (int)(sk[k] & 0xffffffffu);
            float4 w = xw[atom];
            perm[slot] = atom;
            pos[atom] = slot;
            xref[slot] = w;
            xprune[slot] = w;
            lo = make_float4(w.x, w.y, w.z, 0.0f);
            hi = lo;
        } else if (k < nslots) {
            perm[slot] = -1;
            xref[slot] = pad;
            xprune[slot] = pad;
            xq[slot] = pad;
            tsort[slot] = 0;
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
            bbox[2 * (c0 + c)] = lo;
            bbox[2 * (c0 + c) + 1] = hi;
            clus_sys[c0 + c] = csys;
        }
    }
}

}  // namespace

cudaError_t nb_launch_set_system(nb_pairlist *pl, const nb_sys &one, cudaStream_t s) {
    k_set_system<<<1, 32, 0, s>>>(pl->sys, pl->sys_shift, one);
    return cudaGetLastError();
}

cudaError_t nb_launch_grid_sort(nb_pairlist *pl, const float *coords, cudaStream_t s) {
    int n = pl->n_atoms;
    cudaError_t e = cudaMemsetAsync(pl->col_count, 0, sizeof(int) * (size_t)pl->ncol, s);
    if (e != cudaSuccess) return e;
    int bs = 256, gb = (n + bs - 1) / bs;
    k_bin<<<gb, bs, 0, s>>>(n, coords, pl->atom_sys, pl->sys, pl->col_count, pl->atom_col, pl->atom_slot, pl->xw,
                            pl->st);
    k_col_scan<<<1, 1024, 0, s>>>(pl->ncol, pl->col_count, pl->col_atom_start, pl->col_clus_start, pl->st);
    k_col_scatter<<<gb, bs, 0, s>>>(n, pl->xw, pl->atom_col, pl->atom_slot, pl->col_atom_start, pl->keys);
    k_col_sort<<<pl->ncol, 256, 0, s>>>(pl->col_count, pl->col_atom_start, pl->col_clus_start, pl->keys, pl->xw,
                                        pl->col_sys, pl->perm, pl->pos, pl->xref, pl->xprune, pl->xq, pl->tsort,
                                        pl->bbox, pl->clus_sys, pl->sys, pl->ztab);
    return cudaGetLastError();
}
