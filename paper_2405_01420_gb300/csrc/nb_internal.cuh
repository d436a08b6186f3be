// Internal declarations of the nonbonded library: pair-list layout in HBM,
// device state, FP32 position contract and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nb.h"

#define NB_CLUSTER 8            // atoms per cluster (i and j)
#define NB_MAX_COL_ATOMS 4096   // atoms per grid column the per-column sort can hold
#define NB_MAX_TYPES 32         // LJ types (table of ntype^2 float4 in shared memory)
#define NB_CI_EXCL_BUF 256      // exclusions within one i-cluster
#define NB_SHIFT_CENTER 13      // shift index of S = (0, 0, 0)
#define NB_LEN_BINS 512         // list-length histogram bins (lengths >= 511 share the last)
#define NB_ZBINS 32             // z bins of a grid column's index of its clusters (ztab)
// The grid sort and the search chain their kernels by programmatic dependent launch for lists of
// up to this many clusters: there it hides launch gaps (96,000 atoms: 103.5 -> 98.2 us per search);
// for a 256-box batch of 3.27M atoms the early-resident blocks cost more (1.44 -> 1.51 ms).
#define NB_SEARCH_PDL_MAX_CLUSTERS 65536
#define NB_COULOMB_F 138.935458f

// Device-side state of one pair list (one allocation, zeroed at creation).
// The first three words are laid out as nb_tracker (nb.h), which
// nb_tracker_enqueue copies to the host as they are.
struct nb_dev_state {
    unsigned err;                  // sticky NB_DEV_* bits
    unsigned last_d2_search;       // max |y - y_search|^2 (float bits) of the last completed call
    unsigned last_d2_prune;        // max |y - y_prune|^2 (float bits) of the last completed call
    int nc;                        // clusters produced by the last search
    unsigned long long list_count; // outer entries allocated by the last search
    unsigned long long inner_count;// entries kept by the last prune
    unsigned work;                 // work counter of the force kernel
    unsigned work_prune;           // work counter of the prune kernel
    unsigned cur_d2_search;        // the same maxima of the running call
    unsigned cur_d2_prune;
    unsigned long long npairs;     // in-range pairs counted by the last force call
    unsigned excl_count;           // excluded pairs recorded by the last search
    unsigned long long tile_count; // gathered tiles written by the last prune
    unsigned nl_count;             // halves with non-local tiles listed by the last prune (halo split)
};

// Per-system parameters (one entry per independent box). A single-system
// pair list has one entry; a batch has one per system.
struct nb_sys {
    float4 box;        // (Lx, Ly, Lz, 0)
    float inv_sx;      // ncx / Lx: x -> column
    float inv_sy;      // ncy / Ly
    int ncx, ncy;      // xy grid columns of this system
    int col_off;       // first global column of this system
    int atom_off;      // first atom of this system
    int n_atoms;       // atoms of this system
    int pad;
};

// Host handle. Device buffers are sized at creation for n_atoms.
struct nb_pairlist {
    int device;
    int num_sms;
    int n_atoms;
    int nc_max;     // upper bound on clusters: ceil(N/8) + ncol_max
    int ncol_max;   // upper bound on grid columns
    size_t cap;     // list entries per list

    // host copy of what the last search / prune set up
    int searched;
    int has_inner;
    float box[3];
    float rlist;
    float r_inner;
    int ncx, ncy, ncol;
    unsigned flags;                 // nb_config.flags given at creation
    int coul_kind;                  // NB_COUL_EWALD / NB_COUL_RF (nb_set_coulomb)
    float eps_rf;
    unsigned coul_flags;            // NB_COUL_SHIFT | NB_COUL_EXCL_CORR
    int has_excl;                   // the last search had exclusion lists
    int force_threads;              // force kernel launch shape (0 = default), see nb_set_force_shape
    int force_chunk;
    int force_blocks_per_sm;
    cudaEvent_t ev_start, ev_stop;  // optional timing events around the force kernel

    // device buffers
    nb_dev_state *st;
    int *col_count;       // [ncol_max]
    int *col_atom_start;  // [ncol_max + 1]
    int *col_clus_start;  // [ncol_max + 1]
    int *atom_col;        // [N]
    int *atom_slot;       // [N] arrival rank within the column
    float4 *xw;           // [N] wrapped search-frame positions, original order
    unsigned long long *keys;  // [N] (z bits << 32 | atom), column-bucketed
    int *perm;            // [8 nc_max] slot -> atom, -1 = padding
    int *pos;             // [N] atom -> slot
    float4 *xref;         // [8 nc_max] wrapped position at the search
    float4 *xprune;       // [8 nc_max] position at the last prune
    float4 *xq;           // [8 nc_max] (y, q) of the current call
    int *tsort;           // [8 nc_max] LJ type of the current call
    float4 *fsort;        // [8 nc_max] force accumulators, sorted order
    float4 *bbox;         // [2 nc_max] lo (w = real atom count), hi (w = column)
    int *ztab;            // [ncol_max (NB_ZBINS + 1)] per column: the first cluster whose upper z bound
                          // reaches k Lz / NB_ZBINS, k = 0..NB_ZBINS (the column's end for none)
    int4 *outer;          // [cap] (cj, shift, mask lo, mask hi)
    int4 *inner;          // [cap]
    int *ci_start;        // [nc_max] first entry of i-cluster ci (both lists)
    int *ci_len_outer;    // [nc_max]
    int *ci_len_inner;    // [nc_max]
    // systems (a batch of independent boxes; one entry for a single system)
    int nsys;
    int batch;            // created by nb_batch_create (boxes fixed at creation)
    nb_sys *sys;          // [nsys]
    float4 *sys_shift;    // [27 nsys] periodic shift vectors per system and shift index
    int *atom_sys;        // [N] system of each atom
    int *col_sys;         // [ncol_max] system of each grid column
    int *clus_sys;        // [nc_max] system of each cluster
    nb_sys *sys_host;     // host copy of the table [nsys]
    int *len_hist;        // [NB_LEN_BINS] list-length histogram (post-prune sorting)
    int *len_key;         // [nc_max] per-i-cluster work after a prune (gathered tiles, else inner entries)
    int *len_offsets;     // [NB_LEN_BINS]
    int *len_cursor;      // [NB_LEN_BINS]
    int *ci_order;        // [nc_max] i-clusters by decreasing list length
    int sorted;           // ci_order matches the list the forces will use
    int sort_pending;     // the last search's list is sorted by length at its first use (unless a prune
                          // comes first and sorts its own)
    int *vt_slot;         // [2 cap * 8] gathered tiles: j slot | shift << 27
    unsigned *vt_mask;    // [2 cap] 4 x 8 in-range bits per gathered tile
    int *half_start;      // [2 parts][2 nc_max] first gathered tile of each half i-cluster
    int *half_len;        // [2 parts][2 nc_max]
    int *nl_list;         // [2 nc_max] halves (2 ci + h) with non-local tiles, from the last prune with a halo
    int n_home;           // atoms [0, n_home) are home atoms (nb_set_home); n_atoms = no halo
    int vt_parts;         // regions of gathered tiles: 1, or 2 (local, non-local) with a halo
    unsigned char *clus_home;  // [nc_max] bit b: slot b of the cluster holds a home atom (with a halo)
    int2 *excl_pairs;     // [excl_cap] excluded pairs (slot_i, slot_j), i < j, of the last search
    size_t excl_cap;
    int has_vtiles;       // the last prune built gathered tiles
    float4 *gsort;        // [8 nc_max] dL/dF in cluster order (adjoint)
    float4 *bsort;        // [8 nc_max] adjoint accumulators (dL/dx, dL/dq)
    double *glj_acc;      // [NB_MAX_TYPES^2 * 2] adjoint LJ accumulators
};

// ---------------------------------------------------------------------------
// FP32 position contract. Every operation is written with explicit
// round-to-nearest intrinsics so that the compiler cannot contract or
// reorder it; the same sequence defines which pairs are within a radius.
// ---------------------------------------------------------------------------

// Wrap a coordinate into [0, L).
__device__ __forceinline__ float nb_wrap(float x, float L) {
    float w = __fsub_rn(x, __fmul_rn(L, floorf(__fdiv_rn(x, L))));
    if (w < 0.0f) w = __fadd_rn(w, L);
    if (w >= L) w = __fsub_rn(w, L);
    if (!(w >= 0.0f && w < L)) w = 0.0f;
    return w;
}

// Image of x nearest to the search-time wrapped position w0.
__device__ __forceinline__ float nb_image(float x, float w0, float L) {
    float k = rintf(__fdiv_rn(__fsub_rn(x, w0), L));
    return __fsub_rn(x, __fmul_rn(k, L));
}

// Squared distance of a displacement, fixed FMA order.
__device__ __forceinline__ float nb_r2(float dx, float dy, float dz) {
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Shift index s = (sx+1)*9 + (sy+1)*3 + (sz+1) -> integer components.
__device__ __forceinline__ int nb_shift_x(int s) { return s / 9 - 1; }
__device__ __forceinline__ int nb_shift_y(int s) { return (s / 3) % 3 - 1; }
__device__ __forceinline__ int nb_shift_z(int s) { return s % 3 - 1; }

// Padding slots sit far from every real atom so that no distance test
// near them passes even before the mask removes them.
#define NB_PAD_COORD (-1.0e6f)

// Records a message for nb_last_error() and returns code (nb_api.cu).
int nb_record_error(int code, const char *msg);

// ---------------------------------------------------------------------------
// Work items per unit (an i-cluster or a half cluster) of the force and
// adjoint kernels: 1 when the grid has no more warps than there are units,
// else up to NB_MAX_SPLIT, so that a small system still reaches every SM
// (each unit's list is then split into nseg ranges, one work item each).
// Splitting larger systems to shorten the launch's tail costs more than it
// saves: every piece repeats the row setup and the reductions. The kernels
// take the unit count from the device (the clusters of the last search).
#define NB_MAX_SPLIT 8
__host__ __device__ inline unsigned nb_work_split(unsigned grid_warps, unsigned units) {
    if (units == 0u) return 1u;
    const unsigned k = grid_warps / units;
    return k < 1u ? 1u : (k > NB_MAX_SPLIT ? NB_MAX_SPLIT : k);
}

// Range [r0, r1) of piece seg of nseg of a range of len items (32-bit; no
// division when nseg is 1, the case of every system large enough to fill
// the GPU).
__device__ __forceinline__ void nb_piece(int len, unsigned seg, unsigned nseg, int &r0, int &r1) {
    if (nseg == 1u) {
        r0 = 0;
        r1 = len;
    } else {
        r0 = (int)(((unsigned)len * seg) / nseg);
        r1 = (int)(((unsigned)len * (seg + 1u)) / nseg);
    }
}

// Programmatic dependent launch. A kernel launched with nb_launch_pdl may be
// scheduled while the work before it in the stream is still running: its
// blocks fill SMs that the predecessor's tail leaves idle, so the launch
// latency between dependent kernels is hidden. Such a kernel starts with
// nb_pdl_wait() (the predecessor has completed and its writes are visible;
// nothing is read or written before it) and then nb_pdl_release(), which
// lets its own successor be scheduled once all of its blocks have started.
// Both are no-ops for a kernel launched the usual way.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void nb_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void nb_pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// nb_launch_if(pdl, ...) launches the usual way when pdl is false.
template <typename... KArgs, typename... Args>
cudaError_t nb_launch_if(bool pdl, void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                         Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
cudaError_t nb_launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                          Args... args) {
    return nb_launch_if(true, kernel, grid, block, smem, s, args...);
}

// ---------------------------------------------------------------------------
// Launchers (return cudaError_t of the launch).
// ---------------------------------------------------------------------------
// one: the system table of a single-system list, written by the first kernel (NULL for a batch,
// whose table is uploaded when it is created)
cudaError_t nb_launch_grid_sort(nb_pairlist *pl, const float *coords, const nb_sys *one, cudaStream_t s);
cudaError_t nb_launch_search(nb_pairlist *pl, const int *excl_off, const int *excl_idx, float rl2,
                             float rl_col, cudaStream_t s);
// part: NB_PART_ALL (every atom), NB_PART_LOCAL (home atoms; zeroes the
// accumulators and energies), NB_PART_NONLOCAL (halo atoms only).
// snapshot: the gather of a prune (records the prune positions and, when
// lists are sorted, clears the list-length histogram).
cudaError_t nb_launch_gather(nb_pairlist *pl, const float *coords, const float *q, const int *type,
                             int ntype, int snapshot, double *energies, int part, cudaStream_t s);
// clus_home[c] bit b = slot b of cluster c holds a home atom (after the grid sort of a search).
cudaError_t nb_launch_clus_home(nb_pairlist *pl, cudaStream_t s);
cudaError_t nb_launch_prune(nb_pairlist *pl, float r_inner2, float stale_search2, cudaStream_t s);
// Orders i-clusters by decreasing ci_len. hist_ready: the histogram of
// ci_len is already in len_hist (the prune computes it), else it is built here.
cudaError_t nb_launch_sort_by_length(nb_pairlist *pl, const int *ci_len, bool hist_ready, cudaStream_t s);
// Clears the list-length histogram ahead of a prune that fills it.
cudaError_t nb_clear_len_hist(nb_pairlist *pl, cudaStream_t s);
// Records the excluded pairs of the caller's exclusion lists as slot pairs
// (after the grid sort, during the search call).
cudaError_t nb_launch_excl_list(nb_pairlist *pl, const int *excl_off, const int *excl_idx, cudaStream_t s);
// Excluded-pair correction (NB_COUL_EXCL_CORR): forces and E_coul, and its adjoint.
cudaError_t nb_launch_excl_corr(nb_pairlist *pl, float rc, float beta, double *energies, cudaStream_t s);
cudaError_t nb_launch_excl_corr_adj(nb_pairlist *pl, float rc, float beta, cudaStream_t s);
cudaError_t nb_launch_backward_vt(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                                  float stale_prune2, cudaStream_t s);
// Force kernels for one part (NB_PART_*). A local part leaves the
// displacement tracker's running maxima for the non-local part, which ends
// the evaluation.
cudaError_t nb_launch_force_vt(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                               double *energies, float stale_prune2, int part, cudaStream_t s);
cudaError_t nb_launch_force(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                            double *energies, float stale_search2, float stale_prune2, int part,
                            cudaStream_t s);
cudaError_t nb_launch_scatter(nb_pairlist *pl, float *forces, cudaStream_t s);
cudaError_t nb_launch_backward(nb_pairlist *pl, int ntype, const float *ljparams, float rc, float beta,
                               const float *g, float *grad_x, float *grad_q, double *grad_lj,
                               float stale_search2, float stale_prune2, cudaStream_t s);
