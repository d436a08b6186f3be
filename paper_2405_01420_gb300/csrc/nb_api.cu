// C ABI of the nonbonded library (declared in include/nb.h): argument
// checks, device buffer ownership, grid sizing and the order of launches.
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nb_internal.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int ok() {
    g_err.clear();
    return NB_OK;
}

#define NB_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail(NB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Makes the pair list's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

void free_buffers(nb_pairlist *pl) {
    void *bufs[] = {pl->st,     pl->col_count, pl->col_atom_start, pl->col_clus_start, pl->atom_col,
                    pl->atom_slot, pl->xw,     pl->keys,           pl->perm,           pl->pos,
                    pl->xref,   pl->xprune,    pl->xq,             pl->tsort,          pl->fsort,
                    pl->bbox,   pl->outer,     pl->inner,          pl->ci_start,       pl->ci_len_outer,
                    pl->ci_len_inner, pl->gsort,   pl->bsort,          pl->glj_acc,        pl->sys,
                    pl->sys_shift, pl->atom_sys, pl->col_sys,       pl->clus_sys,       pl->len_hist,
                    pl->len_offsets, pl->len_cursor, pl->ci_order,     pl->vt_slot,        pl->vt_mask,
                    pl->half_start, pl->half_len,  pl->len_key,      pl->excl_pairs,  pl->clus_home,
                    pl->ztab,   pl->nl_list};
    for (void *b : bufs)
        if (b) cudaFree(b);
}

template <class T>
bool alloc(T **p, size_t count, size_t *total) {
    size_t bytes = sizeof(T) * (count ? count : 1);
    *total += bytes;
    return cudaMalloc((void **)p, bytes) == cudaSuccess;
}

float sq_nonneg(double x) { return x > 0.0 ? (float)(x * x) : 0.0f; }

// Displacement budget: half the radius difference, less 1e-5 nm so that
// FP32 rounding of the distances cannot use up the margin.
float stale_bound2(double r_big, double r_small) { return sq_nonneg(0.5 * (r_big - r_small) - 1e-5); }



// xy columns of ~cubic 8-atom cells at the mean density of one system,
// at most ncol_cap columns.
void grid_for(double Lx, double Ly, double Lz, double n, long long ncol_cap, int *ncx_out, int *ncy_out) {
    const double side = std::cbrt(NB_CLUSTER * Lx * Ly * Lz / n);
    int ncx = std::max(1, (int)std::floor(Lx / side));
    int ncy = std::max(1, (int)std::floor(Ly / side));
    while (n / ((double)ncx * ncy) > NB_MAX_COL_ATOMS / 4 && (long long)(ncx + 1) * (ncy + 1) <= ncol_cap) {
        ++ncx;
        ++ncy;
    }
    while ((long long)ncx * ncy > ncol_cap) {
        if (ncx >= ncy) --ncx; else --ncy;
    }
    *ncx_out = ncx;
    *ncy_out = ncy;
}

nb_sys make_sys(const float *box, int ncx, int ncy, int col_off, int atom_off, int n_atoms) {
    nb_sys S;
    std::memset(&S, 0, sizeof(S));
    S.box = make_float4(box[0], box[1], box[2], 0.0f);
    S.inv_sx = (float)(ncx / (double)box[0]);
    S.inv_sy = (float)(ncy / (double)box[1]);
    S.ncx = ncx;
    S.ncy = ncy;
    S.col_off = col_off;
    S.atom_off = atom_off;
    S.n_atoms = n_atoms;
    return S;
}

// Allocates every device buffer of a pair list over n atoms in nsys systems.
int alloc_pairlist(nb_pairlist *pl, long long n, const nb_config *cfg, const char *who) {
    if (cfg && (cfg->flags & ~(unsigned)(NB_FLAG_COUNT_PAIRS | NB_FLAG_NO_LIST_SORT | NB_FLAG_CLUSTER_TILES)) != 0u)
        return fail(NB_ERR_ARG, "%s: unknown flags 0x%x", who, cfg->flags);
    NB_CUDA(cudaGetDevice(&pl->device));
    NB_CUDA(cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device));
    const long long nclus = (n + NB_CLUSTER - 1) / NB_CLUSTER;
    pl->n_atoms = (int)n;
    size_t cap = (cfg && cfg->capacity_entries) ? cfg->capacity_entries : (size_t)nclus * 200 + 65536;
    if (cap >= (size_t)1 << 31) return fail(NB_ERR_ARG, "%s: capacity_entries %zu >= 2^31", who, cap);
    pl->cap = cap;
    pl->excl_cap = 8 * (size_t)n + 64;  // excluded pairs (i < j): 8 per atom
    pl->n_home = n;                     // no halo until nb_set_home
    pl->vt_parts = 1;
    pl->flags = cfg ? cfg->flags : 0u;
    // one extra cluster of slots past the last cluster: slot 8 nc_max pads
    // the last gathered tile of a half and never holds an atom
    const size_t nslot = (size_t)pl->nc_max * NB_CLUSTER + NB_CLUSTER;
    size_t total = 0;
    bool good = alloc(&pl->st, 1, &total) && alloc(&pl->col_count, pl->ncol_max, &total) &&
                alloc(&pl->col_atom_start, pl->ncol_max + 1, &total) &&
                alloc(&pl->col_clus_start, pl->ncol_max + 1, &total) && alloc(&pl->atom_col, n, &total) &&
                alloc(&pl->atom_slot, n, &total) && alloc(&pl->xw, n, &total) && alloc(&pl->keys, n, &total) &&
                alloc(&pl->perm, nslot, &total) && alloc(&pl->pos, n, &total) && alloc(&pl->xref, nslot, &total) &&
                alloc(&pl->xprune, nslot, &total) && alloc(&pl->xq, nslot, &total) &&
                alloc(&pl->tsort, nslot, &total) && alloc(&pl->fsort, nslot, &total) &&
                alloc(&pl->bbox, 2 * (size_t)pl->nc_max, &total) && alloc(&pl->outer, cap, &total) &&
                alloc(&pl->inner, cap, &total) && alloc(&pl->ci_start, pl->nc_max, &total) &&
                alloc(&pl->ci_len_outer, pl->nc_max, &total) && alloc(&pl->ci_len_inner, pl->nc_max, &total) &&
                alloc(&pl->gsort, nslot, &total) && alloc(&pl->bsort, nslot, &total) &&
                alloc(&pl->glj_acc, 2 * NB_MAX_TYPES * NB_MAX_TYPES, &total) && alloc(&pl->sys, pl->nsys, &total) &&
                alloc(&pl->sys_shift, 27 * (size_t)pl->nsys, &total) && alloc(&pl->atom_sys, n, &total) &&
                alloc(&pl->col_sys, pl->ncol_max, &total) && alloc(&pl->clus_sys, pl->nc_max, &total) &&
                alloc(&pl->len_hist, NB_LEN_BINS, &total) && alloc(&pl->len_offsets, NB_LEN_BINS, &total) &&
                alloc(&pl->len_cursor, NB_LEN_BINS, &total) && alloc(&pl->ci_order, pl->nc_max, &total) &&
                alloc(&pl->len_key, pl->nc_max, &total) &&
                alloc(&pl->excl_pairs, pl->excl_cap, &total) &&
                alloc(&pl->half_start, 4 * (size_t)pl->nc_max, &total) &&
                alloc(&pl->half_len, 4 * (size_t)pl->nc_max, &total) &&
                alloc(&pl->nl_list, 2 * (size_t)pl->nc_max, &total) &&
                alloc(&pl->clus_home, (size_t)pl->nc_max, &total) &&
                alloc(&pl->ztab, (size_t)pl->ncol_max * (NB_ZBINS + 1), &total);
    // gathered tiles pack a slot in 27 bits and index tiles with 32-bit ints;
    // beyond that the force kernel stays on the cluster-pair tiles
    if (good && nslot < ((size_t)1 << 27) && 2 * cap < ((size_t)1 << 31))
        good = alloc(&pl->vt_slot, 16 * cap, &total) && alloc(&pl->vt_mask, 2 * cap, &total);
    if (!good) {
        cudaGetLastError();  // clear the allocation error
        return fail(NB_ERR_NOMEM, "%s: cudaMalloc of %zu bytes failed", who, total);
    }
    pl->sys_host = new (std::nothrow) nb_sys[pl->nsys];
    if (!pl->sys_host) return fail(NB_ERR_NOMEM, "%s: host allocation failed", who);
    // Defined contents for everything a kernel may read before the first search writes it.
    NB_CUDA(cudaMemset(pl->st, 0, sizeof(nb_dev_state)));
    NB_CUDA(cudaMemset(pl->pos, 0, sizeof(int) * (size_t)n));
    NB_CUDA(cudaMemset(pl->perm, 0xff, sizeof(int) * nslot));
    NB_CUDA(cudaMemset(pl->ci_start, 0, sizeof(int) * (size_t)pl->nc_max));
    NB_CUDA(cudaMemset(pl->ci_len_outer, 0, sizeof(int) * (size_t)pl->nc_max));
    NB_CUDA(cudaMemset(pl->ci_len_inner, 0, sizeof(int) * (size_t)pl->nc_max));
    NB_CUDA(cudaMemset(pl->fsort, 0, sizeof(float4) * nslot));
    NB_CUDA(cudaMemset(pl->atom_sys, 0, sizeof(int) * (size_t)n));
    NB_CUDA(cudaMemset(pl->col_sys, 0, sizeof(int) * (size_t)pl->ncol_max));
    NB_CUDA(cudaMemset(pl->clus_sys, 0, sizeof(int) * (size_t)pl->nc_max));
    NB_CUDA(cudaMemset(pl->tsort, 0, sizeof(int) * nslot));
    NB_CUDA(cudaMemset(pl->gsort, 0, sizeof(float4) * nslot));  // the pad slot's g stays 0
    const float4 far = make_float4(NB_PAD_COORD, NB_PAD_COORD, NB_PAD_COORD, 0.0f);
    NB_CUDA(cudaMemcpy(pl->xq + (size_t)pl->nc_max * NB_CLUSTER, &far, sizeof(float4), cudaMemcpyHostToDevice));
    return NB_OK;
}

void destroy_partial(nb_pairlist *pl) {
    free_buffers(pl);
    delete[] pl->sys_host;
    delete pl;
}

}  // namespace

int nb_record_error(int code, const char *msg) { return fail(code, "%s", msg); }

extern "C" const char *nb_version(void) { return "nb 0.1.0 sm_103a"; }

extern "C" const char *nb_last_error(void) { return g_err.c_str(); }

extern "C" int nb_pairlist_create(nb_pairlist **out, int n_atoms, const nb_config *cfg) {
    if (!out) return fail(NB_ERR_ARG, "nb_pairlist_create: out is NULL");
    *out = nullptr;
    if (n_atoms < 1) return fail(NB_ERR_ARG, "nb_pairlist_create: n_atoms = %d < 1", n_atoms);
    nb_pairlist *pl = new (std::nothrow) nb_pairlist;
    if (!pl) return fail(NB_ERR_NOMEM, "nb_pairlist_create: host allocation failed");
    std::memset(pl, 0, sizeof(*pl));
    const long long nclus = ((long long)n_atoms + NB_CLUSTER - 1) / NB_CLUSTER;
    pl->nsys = 1;
    pl->ncol_max = (int)nclus;
    pl->nc_max = (int)(nclus + pl->ncol_max);
    const int rc = alloc_pairlist(pl, n_atoms, cfg, "nb_pairlist_create");
    if (rc != NB_OK) {
        destroy_partial(pl);
        return rc;
    }
    NB_CUDA(cudaDeviceSynchronize());
    *out = pl;
    return ok();
}

extern "C" int nb_batch_create(nb_pairlist **out, int n_systems, const int *atom_off, const float *boxes,
                               const nb_config *cfg) {
    if (!out || !atom_off || !boxes) return fail(NB_ERR_ARG, "nb_batch_create: NULL argument");
    *out = nullptr;
    if (n_systems < 1) return fail(NB_ERR_ARG, "nb_batch_create: n_systems = %d < 1", n_systems);
    if (atom_off[0] != 0) return fail(NB_ERR_ARG, "nb_batch_create: atom_off[0] must be 0");
    for (int b = 0; b < n_systems; ++b) {
        if (atom_off[b + 1] <= atom_off[b]) return fail(NB_ERR_ARG, "nb_batch_create: system %d has no atoms", b);
        for (int k = 0; k < 3; ++k)
            if (!(boxes[3 * b + k] > 0.0f) || !std::isfinite(boxes[3 * b + k]))
                return fail(NB_ERR_ARG, "nb_batch_create: bad box edge for system %d", b);
    }
    const long long n = atom_off[n_systems];
    std::vector<nb_sys> sys(n_systems);
    long long ncol = 0, ncl = 0;
    for (int b = 0; b < n_systems; ++b) {
        const long long nb = atom_off[b + 1] - atom_off[b];
        const long long cap_cols = (nb + NB_CLUSTER - 1) / NB_CLUSTER;
        int ncx, ncy;
        grid_for(boxes[3 * b], boxes[3 * b + 1], boxes[3 * b + 2], (double)nb, cap_cols, &ncx, &ncy);
        sys[b] = make_sys(boxes + 3 * b, ncx, ncy, (int)ncol, atom_off[b], (int)nb);
        ncol += (long long)ncx * ncy;
        ncl += cap_cols;
    }
    if (n + ncol + ncl >= ((long long)1 << 28)) return fail(NB_ERR_ARG, "nb_batch_create: batch too large");
    nb_pairlist *pl = new (std::nothrow) nb_pairlist;
    if (!pl) return fail(NB_ERR_NOMEM, "nb_batch_create: host allocation failed");
    std::memset(pl, 0, sizeof(*pl));
    pl->nsys = n_systems;
    pl->batch = 1;
    pl->ncol_max = (int)ncol;
    pl->ncol = (int)ncol;
    pl->nc_max = (int)(ncl + ncol);
    int rc = alloc_pairlist(pl, n, cfg, "nb_batch_create");
    if (rc == NB_OK) {
        std::vector<float4> shift(27 * (size_t)n_systems);
        std::vector<int> atom_sys(n), col_sys(ncol);
        for (int b = 0; b < n_systems; ++b) {
            pl->sys_host[b] = sys[b];
            for (int k = 0; k < 27; ++k)
                shift[27 * b + k] = make_float4((float)((k / 9) - 1) * boxes[3 * b], (float)(((k / 3) % 3) - 1) * boxes[3 * b + 1],
                                                (float)((k % 3) - 1) * boxes[3 * b + 2], 0.0f);
            for (int i = atom_off[b]; i < atom_off[b + 1]; ++i) atom_sys[i] = b;
            for (int c = 0; c < sys[b].ncx * sys[b].ncy; ++c) col_sys[sys[b].col_off + c] = b;
        }
        if (cudaMemcpy(pl->sys, sys.data(), sizeof(nb_sys) * n_systems, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->sys_shift, shift.data(), sizeof(float4) * shift.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->atom_sys, atom_sys.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(pl->col_sys, col_sys.data(), sizeof(int) * ncol, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            rc = fail(NB_ERR_CUDA, "nb_batch_create: upload of the system table failed");
    }
    if (rc != NB_OK) {
        destroy_partial(pl);
        return rc;
    }
    *out = pl;
    return ok();
}

extern "C" int nb_pairlist_destroy(nb_pairlist *pl) {
    if (!pl) return ok();
    DeviceGuard g(pl->device);
    cudaDeviceSynchronize();
    free_buffers(pl);
    delete[] pl->sys_host;
    delete pl;
    return ok();
}

extern "C" int nb_search(nb_pairlist *pl, const float *coords, const float *box, float rlist,
                         const int *excl_off, const int *excl_idx, void *stream) {
    if (!pl || !coords) return fail(NB_ERR_ARG, "nb_search: NULL pair list or coords");
    if (pl->batch && box)
        return fail(NB_ERR_ARG, "nb_search: the boxes of a batch are fixed at nb_batch_create; pass box = NULL");
    if (!pl->batch && !box) return fail(NB_ERR_ARG, "nb_search: box is NULL");
    if ((excl_off == nullptr) != (excl_idx == nullptr))
        return fail(NB_ERR_ARG, "nb_search: excl_off and excl_idx must both be given or both NULL");
    if (!(rlist > 0.0f) || !std::isfinite(rlist)) return fail(NB_ERR_ARG, "nb_search: rlist = %g", rlist);
    const float *boxes = pl->batch ? nullptr : box;
    float lmax = 0.0f;
    for (int b = 0; b < pl->nsys; ++b) {
        float L[3];
        for (int k = 0; k < 3; ++k) {
            L[k] = boxes ? boxes[k] : (k == 0 ? pl->sys_host[b].box.x : (k == 1 ? pl->sys_host[b].box.y : pl->sys_host[b].box.z));
            if (!std::isfinite(L[k]) || !(L[k] > 2.0f * rlist))
                return fail(NB_ERR_ARG, "nb_search: box edge %g (system %d) must exceed 2*rlist = %g", L[k], b,
                            2.0f * rlist);
            lmax = std::max(lmax, L[k]);
        }
    }
    DeviceGuard g(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!pl->batch) {
        for (int k = 0; k < 3; ++k) pl->box[k] = box[k];
        int ncx, ncy;
        grid_for(box[0], box[1], box[2], (double)pl->n_atoms, pl->ncol_max, &ncx, &ncy);
        pl->ncx = ncx;
        pl->ncy = ncy;
        pl->ncol = ncx * ncy;
        pl->sys_host[0] = make_sys(box, ncx, ncy, 0, 0, pl->n_atoms);
    }
    // the grid sort's first kernel clears the list counter (and writes a single system's table)
    NB_CUDA(nb_launch_grid_sort(pl, coords, pl->batch ? nullptr : &pl->sys_host[0], s));

    // The bounding-box test uses a radius inflated by a few ulps of the box
    // edge, so that every pair within rlist under the FP32 distance contract
    // is in the list (the list is a buffered superset anyway).
    const double ulp = (double)std::nextafter(lmax, 2.0f * lmax) - lmax;
    const double rle = rlist + std::max(1e-5, 8.0 * ulp) + 1e-6 * rlist;
    const float rl2 = std::nextafter((float)(rle * rle), 1e30f);
    const float rl_col = (float)(rle + 1e-3);
    NB_CUDA(nb_launch_search(pl, excl_off, excl_idx, rl2, rl_col, s));
    if (pl->vt_parts == 2) NB_CUDA(nb_launch_clus_home(pl, s));  // home bits of the clusters (a halo)
    // the excluded pairs, as slot pairs, for the excluded-pair correction (only when it is on: the
    // caller's lists are read only during this call)
    pl->has_excl = excl_off != nullptr && (pl->coul_flags & NB_COUL_EXCL_CORR);
    if (pl->has_excl) {
        NB_CUDA(cudaMemsetAsync(&pl->st->excl_count, 0, sizeof(unsigned), s));
        NB_CUDA(nb_launch_excl_list(pl, excl_off, excl_idx, s));
    }
    // ordering the clusters by list length waits for the first force or adjoint call on this list: a
    // prune that comes first orders them by its own (pruned) work instead
    pl->sorted = 0;
    // A system small enough that the force kernel splits every list four ways or more has no
    // launch tail for the ordering to shorten: its three kernels would only add latency.
    const bool small = (long long)pl->nc_max * 4 <= (long long)pl->num_sms * 32;
    pl->sort_pending = !(pl->flags & NB_FLAG_NO_LIST_SORT) && !small;
    pl->searched = 1;
    pl->has_inner = 0;
    pl->has_vtiles = 0;
    pl->rlist = rlist;
    pl->r_inner = 0.0f;
    return ok();
}

// Orders the i-clusters of a search's list by length if that is still due.
static cudaError_t sort_if_pending(nb_pairlist *pl, cudaStream_t s) {
    if (!pl->sort_pending) return cudaSuccess;
    pl->sort_pending = 0;
    if (pl->flags & NB_FLAG_NO_LIST_SORT) return cudaSuccess;
    const cudaError_t e = nb_launch_sort_by_length(pl, pl->ci_len_outer, false, s);
    if (e == cudaSuccess) pl->sorted = 1;
    return e;
}

extern "C" int nb_prune(nb_pairlist *pl, const float *coords, float r_inner, void *stream) {
    if (!pl || !coords) return fail(NB_ERR_ARG, "nb_prune: NULL pair list or coords");
    if (!pl->searched) return fail(NB_ERR_STATE, "nb_prune: no search yet");
    if (!(r_inner > 0.0f) || !(r_inner <= pl->rlist))
        return fail(NB_ERR_ARG, "nb_prune: r_inner = %g must be in (0, rlist = %g]", r_inner, pl->rlist);
    DeviceGuard g(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    // the snapshot gather also clears the list-length histogram that the prune fills
    NB_CUDA(nb_launch_gather(pl, coords, nullptr, nullptr, 1, 1, nullptr, NB_PART_ALL, s));
    const float r2cut = r_inner * r_inner;
    const bool sort = !(pl->flags & NB_FLAG_NO_LIST_SORT);
    NB_CUDA(nb_launch_prune(pl, r2cut, stale_bound2(pl->rlist, r_inner), s));
    pl->sorted = 0;
    pl->sort_pending = 0;
    if (sort) {
        NB_CUDA(nb_launch_sort_by_length(pl, pl->len_key, true, s));
        pl->sorted = 1;
    }
    pl->has_inner = 1;
    pl->has_vtiles = pl->vt_slot != nullptr;
    pl->r_inner = r_inner;
    return ok();
}

// nb_forces and nb_forces_part; `who` names the entry point in error messages.
static int forces_impl(const char *who, nb_pairlist *pl, int part, const float *coords, const float *q,
                       const int *type, int ntype, const float *ljparams, float rc, float beta, float *forces,
                       double *energies, void *stream) {
    if (part != NB_PART_ALL && part != NB_PART_LOCAL && part != NB_PART_NONLOCAL)
        return fail(NB_ERR_ARG, "%s: part = %d", who, part);
    if (!pl || !coords || !q || !type || !ljparams || (!forces && part != NB_PART_LOCAL))
        return fail(NB_ERR_ARG, "%s: NULL argument", who);
    if (!pl->searched) return fail(NB_ERR_STATE, "%s: no search yet", who);
    if (ntype < 1 || ntype > NB_MAX_TYPES)
        return fail(NB_ERR_ARG, "%s: ntype = %d not in [1, %d]", who, ntype, NB_MAX_TYPES);
    const float rmax = pl->has_inner ? pl->r_inner : pl->rlist;
    if (!(rc > 0.0f) || !(rc <= rmax))
        return fail(NB_ERR_ARG, "%s: rc = %g must be in (0, %g] (list radius)", who, rc, rmax);
    if (pl->coul_kind == NB_COUL_EWALD && (!(beta >= 0.0f) || !((double)beta * rc <= 3.2)))
        return fail(NB_ERR_ARG, "%s: beta*rc = %g must be in [0, 3.2]", who, (double)beta * rc);
    if ((pl->coul_flags & NB_COUL_EXCL_CORR) && !pl->has_excl)
        return fail(NB_ERR_STATE, "%s: NB_COUL_EXCL_CORR needs a search with exclusion lists made while it was set",
                    who);
    DeviceGuard g(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    // Without a halo the local part is the whole computation and the
    // non-local part only writes the forces.
    const bool split = pl->vt_parts == 2;
    const bool compute = split || part != NB_PART_NONLOCAL;
    const int kpart = split ? part : NB_PART_ALL;
    const bool last = part != NB_PART_LOCAL;  // this call ends the evaluation
    if (compute) {
        NB_CUDA(sort_if_pending(pl, s));
        NB_CUDA(nb_launch_gather(pl, coords, q, type, ntype, 0, energies, kpart, s));
        if (pl->ev_start) NB_CUDA(cudaEventRecord(pl->ev_start, s));
        const int fpart = (!split && part == NB_PART_LOCAL) ? NB_PART_ALL : kpart;
        if (pl->has_vtiles && !(pl->flags & NB_FLAG_CLUSTER_TILES))
            NB_CUDA(nb_launch_force_vt(pl, ntype, ljparams, rc, beta, energies, stale_bound2(pl->r_inner, rc), fpart,
                                       s));
        else
            NB_CUDA(nb_launch_force(pl, ntype, ljparams, rc, beta, energies, stale_bound2(pl->rlist, rc),
                                    stale_bound2(pl->r_inner, rc), fpart, s));
        if (pl->ev_stop) NB_CUDA(cudaEventRecord(pl->ev_stop, s));
    }
    if (last) {
        if (pl->coul_flags & NB_COUL_EXCL_CORR) NB_CUDA(nb_launch_excl_corr(pl, rc, beta, energies, s));
        NB_CUDA(nb_launch_scatter(pl, forces, s));
    }
    return ok();
}

extern "C" int nb_forces_part(nb_pairlist *pl, int part, const float *coords, const float *q, const int *type,
                              int ntype, const float *ljparams, float rc, float beta, float *forces, double *energies,
                              void *stream) {
    return forces_impl("nb_forces_part", pl, part, coords, q, type, ntype, ljparams, rc, beta, forces, energies,
                       stream);
}

extern "C" int nb_forces(nb_pairlist *pl, const float *coords, const float *q, const int *type, int ntype,
                         const float *ljparams, float rc, float beta, float *forces, double *energies,
                         void *stream) {
    return forces_impl("nb_forces", pl, NB_PART_ALL, coords, q, type, ntype, ljparams, rc, beta, forces, energies,
                       stream);
}

extern "C" int nb_backward(nb_pairlist *pl, const float *coords, const float *q, const int *type, int ntype,
                           const float *ljparams, float rc, float beta, const float *g, float *grad_x,
                           float *grad_q, double *grad_lj, void *stream) {
    if (!pl || !coords || !q || !type || !ljparams || !g || !grad_x || !grad_q || !grad_lj)
        return fail(NB_ERR_ARG, "nb_backward: NULL argument");
    if (!pl->searched) return fail(NB_ERR_STATE, "nb_backward: no search yet");
    if (ntype < 1 || ntype > NB_BACKWARD_MAX_TYPES)
        return fail(NB_ERR_ARG, "nb_backward: ntype = %d not in [1, %d]", ntype, NB_BACKWARD_MAX_TYPES);
    const float rmax = pl->has_inner ? pl->r_inner : pl->rlist;
    if (!(rc > 0.0f) || !(rc <= rmax))
        return fail(NB_ERR_ARG, "nb_backward: rc = %g must be in (0, %g] (list radius)", rc, rmax);
    if (pl->coul_kind == NB_COUL_EWALD && (!(beta >= 0.0f) || !((double)beta * rc <= 3.2)))
        return fail(NB_ERR_ARG, "nb_backward: beta*rc = %g must be in [0, 3.2]", (double)beta * rc);
    if ((pl->coul_flags & NB_COUL_EXCL_CORR) && !pl->has_excl)
        return fail(NB_ERR_STATE, "nb_backward: NB_COUL_EXCL_CORR needs a search with exclusion lists made while it was set");
    DeviceGuard gd(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(sort_if_pending(pl, s));
    NB_CUDA(nb_launch_gather(pl, coords, q, type, ntype, 0, nullptr, NB_PART_ALL, s));
    NB_CUDA(nb_launch_backward(pl, ntype, ljparams, rc, beta, g, grad_x, grad_q, grad_lj,
                               stale_bound2(pl->rlist, rc), stale_bound2(pl->r_inner, rc), s));
    return ok();
}

extern "C" int nb_status(nb_pairlist *pl, unsigned *error_word, int clear, void *stream) {
    if (!pl || !error_word) return fail(NB_ERR_ARG, "nb_status: NULL argument");
    DeviceGuard g(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned w = 0;
    NB_CUDA(cudaMemcpyAsync(&w, &pl->st->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    if (clear) NB_CUDA(cudaMemsetAsync(&pl->st->err, 0, sizeof(unsigned), s));
    NB_CUDA(cudaStreamSynchronize(s));
    *error_word = w;
    return ok();
}

extern "C" int nb_pairlist_stats(nb_pairlist *pl, nb_stats *out, void *stream) {
    if (!pl || !out) return fail(NB_ERR_ARG, "nb_pairlist_stats: NULL argument");
    DeviceGuard g(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    nb_dev_state st;
    NB_CUDA(cudaMemcpyAsync(&st, pl->st, sizeof(st), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    std::memset(out, 0, sizeof(*out));
    out->n_atoms = pl->n_atoms;
    out->n_clusters = pl->searched ? st.nc : 0;
    out->n_columns = pl->searched ? pl->ncol : 0;
    out->has_inner = pl->has_inner;
    out->outer_entries = (long long)st.list_count;
    out->inner_entries = pl->has_inner ? (long long)st.inner_count : 0;
    out->capacity_entries = (long long)pl->cap;
    out->pairs_last = (pl->flags & NB_FLAG_COUNT_PAIRS) ? (long long)st.npairs : -1;
    out->rlist = pl->rlist;
    out->r_inner = pl->r_inner;
    float ds, dp;
    std::memcpy(&ds, &st.last_d2_search, sizeof(float));
    std::memcpy(&dp, &st.last_d2_prune, sizeof(float));
    out->max_disp_search = std::sqrt(ds);
    out->max_disp_prune = std::sqrt(dp);
    out->error_word = st.err;
    out->gathered_tiles = pl->has_vtiles ? (long long)st.tile_count : 0;
    return ok();
}

static_assert(sizeof(nb_tracker) == 3 * sizeof(unsigned), "nb_tracker is three 32-bit words");
static_assert(offsetof(nb_dev_state, err) == offsetof(nb_tracker, error_word) &&
                  offsetof(nb_dev_state, last_d2_search) == offsetof(nb_tracker, max_disp2_search) &&
                  offsetof(nb_dev_state, last_d2_prune) == offsetof(nb_tracker, max_disp2_prune),
              "nb_dev_state starts with the words of nb_tracker");

extern "C" int nb_tracker_enqueue(nb_pairlist *pl, nb_tracker *out, void *stream) {
    if (!pl || !out) return fail(NB_ERR_ARG, "nb_tracker_enqueue: NULL argument");
    DeviceGuard g(pl->device);
    NB_CUDA(cudaMemcpyAsync(out, pl->st, sizeof(nb_tracker), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    return ok();
}

extern "C" int nb_pairlist_export(nb_pairlist *pl, int which, int *ci, int *cj, int *shift,
                                  unsigned long long *mask, size_t cap, size_t *n_out, int *perm,
                                  size_t perm_cap, size_t *n_slots, void *stream) {
    if (!pl || !n_out) return fail(NB_ERR_ARG, "nb_pairlist_export: NULL argument");
    if (cap > 0 && (!ci || !cj || !shift || !mask)) return fail(NB_ERR_ARG, "nb_pairlist_export: NULL output arrays");
    if (which != NB_LIST_OUTER && which != NB_LIST_INNER) return fail(NB_ERR_ARG, "nb_pairlist_export: bad list id %d", which);
    if (!pl->searched) return fail(NB_ERR_STATE, "nb_pairlist_export: no search yet");
    if (which == NB_LIST_INNER && !pl->has_inner) return fail(NB_ERR_STATE, "nb_pairlist_export: no prune since the search");
    DeviceGuard g(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    nb_dev_state st;
    NB_CUDA(cudaMemcpyAsync(&st, pl->st, sizeof(st), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    const int nc = st.nc;
    const size_t used = std::min((size_t)st.list_count, pl->cap);
    std::vector<int> start(nc), len(nc);
    std::vector<int4> ent(used);
    NB_CUDA(cudaMemcpyAsync(start.data(), pl->ci_start, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaMemcpyAsync(len.data(), which == NB_LIST_OUTER ? pl->ci_len_outer : pl->ci_len_inner,
                            sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
    if (used)
        NB_CUDA(cudaMemcpyAsync(ent.data(), which == NB_LIST_OUTER ? pl->outer : pl->inner, sizeof(int4) * used,
                                cudaMemcpyDeviceToHost, s));
    const size_t nslot = (size_t)nc * NB_CLUSTER;
    if (n_slots) *n_slots = nslot;
    if (perm && perm_cap >= nslot)
        NB_CUDA(cudaMemcpyAsync(perm, pl->perm, sizeof(int) * nslot, cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    size_t k = 0;
    for (int c = 0; c < nc; ++c) {
        for (int t = 0; t < len[c]; ++t, ++k) {
            if (k >= cap) continue;
            const size_t idx = (size_t)start[c] + t;
            if (idx >= used) return fail(NB_ERR_STATE, "nb_pairlist_export: entry %zu beyond the list", idx);
            const int4 e = ent[idx];
            ci[k] = c;
            cj[k] = e.x;
            shift[k] = e.y;
            mask[k] = (unsigned long long)(unsigned)e.z | ((unsigned long long)(unsigned)e.w << 32);
        }
    }
    *n_out = k;
    if (perm && perm_cap < nslot) return fail(NB_ERR_CAPACITY, "nb_pairlist_export: perm_cap %zu < %zu slots", perm_cap, nslot);
    if (k > cap) return fail(NB_ERR_CAPACITY, "nb_pairlist_export: %zu entries > cap %zu", k, cap);
    return ok();
}

extern "C" int nb_set_timing_events(nb_pairlist *pl, void *start, void *stop) {
    if (!pl) return fail(NB_ERR_ARG, "nb_set_timing_events: NULL pair list");
    if ((start == nullptr) != (stop == nullptr))
        return fail(NB_ERR_ARG, "nb_set_timing_events: give both events or neither");
    pl->ev_start = (cudaEvent_t)start;
    pl->ev_stop = (cudaEvent_t)stop;
    return ok();
}

extern "C" int nb_set_force_shape(nb_pairlist *pl, int threads, int chunk, int blocks_per_sm) {
    if (!pl) return fail(NB_ERR_ARG, "nb_set_force_shape: NULL pair list");
    if (threads != 0 && threads != 128 && threads != 256)
        return fail(NB_ERR_ARG, "nb_set_force_shape: threads must be 0, 128 or 256");
    if (chunk != 0 && chunk != 8 && chunk != 16) return fail(NB_ERR_ARG, "nb_set_force_shape: chunk must be 0, 8 or 16");
    if (blocks_per_sm < 0) return fail(NB_ERR_ARG, "nb_set_force_shape: blocks_per_sm < 0");
    pl->force_threads = threads;
    pl->force_chunk = chunk;
    pl->force_blocks_per_sm = blocks_per_sm;
    return ok();
}

extern "C" int nb_pairlist_export_tiles(nb_pairlist *pl, int *half_id, int *slots, unsigned *masks, size_t cap,
                                        size_t *n_out, void *stream) {
    if (!pl || !n_out) return fail(NB_ERR_ARG, "nb_pairlist_export_tiles: NULL argument");
    if (cap > 0 && (!half_id || !slots || !masks)) return fail(NB_ERR_ARG, "nb_pairlist_export_tiles: NULL arrays");
    if (!pl->has_vtiles) return fail(NB_ERR_STATE, "nb_pairlist_export_tiles: no prune since the search");
    DeviceGuard g(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    nb_dev_state st;
    NB_CUDA(cudaMemcpyAsync(&st, pl->st, sizeof(st), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    const int nh = 2 * st.nc, nreg = pl->vt_parts == 2 ? 2 : 1;
    std::vector<int> start(nh * nreg), len(nh * nreg);
    for (int r = 0; r < nreg; ++r) {  // regions: local, non-local (with a halo)
        NB_CUDA(cudaMemcpyAsync(start.data() + r * nh, pl->half_start + (size_t)r * 2 * pl->nc_max, sizeof(int) * nh,
                                cudaMemcpyDeviceToHost, s));
        NB_CUDA(cudaMemcpyAsync(len.data() + r * nh, pl->half_len + (size_t)r * 2 * pl->nc_max, sizeof(int) * nh,
                                cudaMemcpyDeviceToHost, s));
    }
    NB_CUDA(cudaStreamSynchronize(s));
    size_t k = 0;
    for (int rh = 0; rh < nh * nreg; ++rh) {
        const int hh = rh % nh;
        const size_t m = (size_t)len[rh];
        if (m > 0 && k + m <= cap) {  // one copy per half: its tiles are contiguous
            NB_CUDA(cudaMemcpyAsync(slots + 8 * k, pl->vt_slot + 8 * (size_t)start[rh], sizeof(int) * 8 * m,
                                    cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaMemcpyAsync(masks + k, pl->vt_mask + start[rh], sizeof(unsigned) * m,
                                    cudaMemcpyDeviceToHost, s));
            for (size_t t = 0; t < m; ++t) half_id[k + t] = hh;
        }
        k += m;
    }
    NB_CUDA(cudaStreamSynchronize(s));
    *n_out = k;
    if (k > cap) return fail(NB_ERR_CAPACITY, "nb_pairlist_export_tiles: %zu tiles > cap %zu", k, cap);
    return ok();
}

extern "C" int nb_set_coulomb(nb_pairlist *pl, int kind, float eps_rf, unsigned flags) {
    if (!pl) return fail(NB_ERR_ARG, "nb_set_coulomb: NULL pair list");
    if (kind != NB_COUL_EWALD && kind != NB_COUL_RF) return fail(NB_ERR_ARG, "nb_set_coulomb: kind = %d", kind);
    if (flags & ~(NB_COUL_SHIFT | NB_COUL_EXCL_CORR)) return fail(NB_ERR_ARG, "nb_set_coulomb: flags = 0x%x", flags);
    if (kind == NB_COUL_RF && (flags & NB_COUL_SHIFT))
        return fail(NB_ERR_ARG, "nb_set_coulomb: NB_COUL_SHIFT is for Ewald (the reaction field is 0 at rc)");
    if (kind == NB_COUL_RF && !(eps_rf == 0.0f || (eps_rf >= 1.0f && std::isfinite(eps_rf))))
        return fail(NB_ERR_ARG, "nb_set_coulomb: eps_rf = %g must be 0 (infinity) or >= 1", eps_rf);
    pl->coul_kind = kind;
    pl->eps_rf = kind == NB_COUL_RF ? eps_rf : 0.0f;
    pl->coul_flags = flags;
    return ok();
}

extern "C" int nb_set_flags(nb_pairlist *pl, unsigned flags) {
    if (!pl) return fail(NB_ERR_ARG, "nb_set_flags: NULL pair list");
    if (flags & ~(unsigned)(NB_FLAG_COUNT_PAIRS | NB_FLAG_NO_LIST_SORT | NB_FLAG_CLUSTER_TILES))
        return fail(NB_ERR_ARG, "nb_set_flags: unknown flags 0x%x", flags);
    pl->flags = flags;
    return ok();
}

extern "C" int nb_set_home(nb_pairlist *pl, int n_home) {
    if (!pl) return fail(NB_ERR_ARG, "nb_set_home: NULL pair list");
    if (pl->batch) return fail(NB_ERR_ARG, "nb_set_home: not for a batch of systems");
    if (n_home < 1 || n_home > pl->n_atoms)
        return fail(NB_ERR_ARG, "nb_set_home: n_home = %d not in [1, %d]", n_home, pl->n_atoms);
    const int parts = n_home < pl->n_atoms ? 2 : 1;
    if (parts == 2 && pl->vt_slot && pl->vt_parts != 2) {
        // the second region of gathered tiles (non-local): twice the buffers
        if (4 * pl->cap >= ((size_t)1 << 31))
            return fail(NB_ERR_CAPACITY, "nb_set_home: list capacity %zu too large for two tile regions", pl->cap);
        DeviceGuard g(pl->device);
        NB_CUDA(cudaDeviceSynchronize());
        int *slot2 = nullptr;
        unsigned *mask2 = nullptr;
        if (cudaMalloc(&slot2, sizeof(int) * 32 * pl->cap) != cudaSuccess ||
            cudaMalloc(&mask2, sizeof(unsigned) * 4 * pl->cap) != cudaSuccess) {
            cudaFree(slot2);
            cudaGetLastError();
            return fail(NB_ERR_NOMEM, "nb_set_home: no memory for the non-local tile region");
        }
        cudaFree(pl->vt_slot);
        cudaFree(pl->vt_mask);
        pl->vt_slot = slot2;
        pl->vt_mask = mask2;
    }
    pl->n_home = n_home;
    pl->vt_parts = parts;
    pl->searched = 0;  // the next nb_search builds the split lists
    pl->has_inner = 0;
    pl->has_vtiles = 0;
    return ok();
}
