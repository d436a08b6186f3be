/*
 * nb.h - C ABI of the GB300 short-range nonbonded library (libnb.so).
 *
 * The library computes short-range nonbonded forces and energies of a
 * periodic particle system: Lennard-Jones plus Ewald real-space Coulomb
 * (erfc) with intra-molecular exclusions, over a cluster-pair (8x8) Verlet
 * list with a rolling prune. This is the "NBNXM" short-range non-bonded
 * kernel that the paper identifies as the rate limiter of a GPU MD step
 * (§III-A, Fig. 2 and the text after it; §IV-A, §IV-B), together with the
 * pair search that feeds it and the prune-only kernel that re-prunes the
 * buffered list ("pair list buffer", "list range", "Prune-only kernel",
 * §III-A). The paper gives no formulas; the arithmetic follows textbook LJ
 * and Ewald real-space physics:
 *
 *   E_LJ = sum_{i<j, not excluded, r < rc} C12_ij/r^12 - C6_ij/r^6
 *                                          - (C12_ij/rc^12 - C6_ij/rc^6)
 *   E_C  = f sum_{i<j, not excluded, r < rc} q_i q_j erfc(beta r)/r
 *   F_i  = -dE/dx_i,   f = 138.935458 kJ mol^-1 nm e^-2
 *
 * Units: nm, e, kJ/mol; forces in kJ mol^-1 nm^-1. Box: orthorhombic,
 * periodic in x, y and z, edges given on the host.
 *
 * Conventions for every function:
 *   - Device pointers are CUDA device addresses owned by the caller; the
 *     library never frees them and keeps no reference after the call
 *     returns, except that launched work reads them until it completes on
 *     the stream. Host pointers are read before the call returns.
 *   - "stream" is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream. Work is stream-ordered; no call synchronises unless
 *     its comment says it does.
 *   - Every function returns NB_OK (0) or an NB_ERR_* code; nb_last_error()
 *     then gives a message (thread-local). Nothing aborts or traps the GPU.
 *     Errors found on the device (list overflow, non-finite coordinates,
 *     a stale list) set bits in a sticky device error word that nb_status()
 *     reads; the forces of a call that set an error bit are not valid.
 *   - A pair list belongs to one device (the current device at creation)
 *     and must be used from one stream at a time.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define NB_OK 0
#define NB_ERR_ARG 1       /* invalid argument (sizes, NULL, box, radii) */
#define NB_ERR_CUDA 2      /* a CUDA runtime call or launch failed */
#define NB_ERR_CAPACITY 3  /* a size exceeds what the pair list was created for */
#define NB_ERR_NONFINITE 4 /* reserved for host-side checks of non-finite input */
#define NB_ERR_TIMEOUT 5   /* reserved: no kernel waits on a flag or another block, so none gives up */
#define NB_ERR_STATE 6     /* call out of order (e.g. nb_forces before nb_search) */
#define NB_ERR_NOMEM 7     /* device allocation failed */

/* Bits of the device error word returned by nb_status(). */
#define NB_DEV_LIST_OVERFLOW 0x01u   /* list entries exceeded capacity_entries */
#define NB_DEV_COLUMN_OVERFLOW 0x02u /* a grid column held more than 4096 atoms */
#define NB_DEV_NONFINITE 0x04u       /* a coordinate was NaN or infinite */
#define NB_DEV_STALE_SEARCH 0x08u    /* atoms moved more than (rlist - r)/2 since the search */
#define NB_DEV_STALE_PRUNE 0x10u     /* atoms moved more than (r_inner - rc)/2 since the prune */
#define NB_DEV_EXCL_OVERFLOW 0x20u   /* >256 exclusions in one 8-atom cluster, an index outside [0, n),
                                        or more than 8 excluded pairs per atom on average */
#define NB_DEV_CLUSTER_OVERFLOW 0x40u /* reserved (not raised: an i-cluster's list length is unbounded) */
#define NB_DEV_BAD_TYPE 0x80u         /* an LJ type outside [0, ntype) (treated as type 0) */

/* Which list nb_pairlist_export() copies. */
#define NB_LIST_OUTER 0 /* built by nb_search at rlist */
#define NB_LIST_INNER 1 /* built by nb_prune at r_inner */

typedef struct nb_pairlist nb_pairlist;

/* Creation options. Zero-initialise and set what you need. */
typedef struct {
    size_t capacity_entries; /* list entries (8x8 cluster pairs) to reserve; 0 = automatic:
                                200 per 8-atom cluster + 65536, enough for rlist <= ~1.3 nm
                                at water density */
    unsigned flags;          /* NB_FLAG_* bits, 0 for none */
} nb_config;

/* nb_config.flags: count the in-range pairs in nb_forces (nb_stats.pairs_last);
   costs about one instruction per pair, so it is off unless asked for. */
#define NB_FLAG_COUNT_PAIRS 0x1u
/* nb_config.flags: do not sort i-clusters by list length after each search
   and prune (§III-A: the post-pruning list sorting that shortens the tail
   of the force kernel; on by default). */
#define NB_FLAG_NO_LIST_SORT 0x2u
/* nb_config.flags: after a prune, compute forces (nb_forces) and the adjoint
   (nb_backward) over the 8x8 cluster-pair tiles of the inner list instead
   of the gathered 4x8 tiles (same results; for comparison). */
#define NB_FLAG_CLUSTER_TILES 0x4u

/* Host-side snapshot of a pair list (filled by nb_pairlist_stats). */
typedef struct {
    int n_atoms;
    int n_clusters;          /* 8-atom clusters after the last search (incl. padding slots) */
    int n_columns;           /* xy grid columns of the last search */
    int has_inner;           /* 1 if nb_prune ran since the last search */
    long long outer_entries; /* cluster pairs in the outer (rlist) list */
    long long inner_entries; /* cluster pairs in the inner (r_inner) list */
    long long capacity_entries;
    long long pairs_last;    /* in-range atom pairs counted by the last nb_forces, or -1 if the
                                pair list was created without NB_FLAG_COUNT_PAIRS */
    float rlist;             /* radius of the last search */
    float r_inner;           /* radius of the last prune (0 if none) */
    float max_disp_search;   /* largest atom displacement since the search, as seen by the last call */
    float max_disp_prune;    /* largest atom displacement since the last prune, as seen by the last call */
    unsigned error_word;     /* sticky device error bits (not cleared by this call) */
    long long gathered_tiles; /* 4 x 8 gathered tiles written by the last prune (32 pair slots each;
                                 0 if none) */
} nb_stats;

/* Library version string, e.g. "nb 0.1.0 sm_103a". */
const char *nb_version(void);

/* Message for the last failing call on this thread ("" if none). */
const char *nb_last_error(void);

/*
 * Create a pair list for systems of exactly n_atoms atoms on the current
 * device. Allocates all device buffers up front (cudaMalloc), so later calls
 * allocate nothing and can be captured in a CUDA graph. cfg may be NULL.
 * Errors: NB_ERR_ARG (n_atoms < 1), NB_ERR_NOMEM, NB_ERR_CUDA.
 */
int nb_pairlist_create(nb_pairlist **pl, int n_atoms, const nb_config *cfg);

/*
 * Create one pair list over a batch of independent systems (boxes), for
 * running many small systems with one set of launches (the batched form of
 * the path; ensemble-style independent systems, §I-A). Systems are stored
 * back to back:
 *   atom_off HOST int[n_systems+1]: system b owns atoms atom_off[b] ..
 *            atom_off[b+1]-1 of every per-atom array (coords, q, type,
 *            forces, ...); atom_off[0] = 0.
 *   boxes    HOST float[3*n_systems]: the orthorhombic box of each system,
 *            fixed for the lifetime of the list.
 * Afterwards nb_search (with box = NULL), nb_prune, nb_forces and
 * nb_backward act on all systems at once; no pair ever joins atoms of two
 * systems. Exclusion indices are global atom indices. nb_forces writes
 * energies as double[2*n_systems] ({E_LJ, E_C} per system). Allocates like
 * nb_pairlist_create and uploads the system table (synchronises once).
 * Errors: NB_ERR_ARG (no systems, empty system, bad box), NB_ERR_NOMEM,
 * NB_ERR_CUDA.
 */
int nb_batch_create(nb_pairlist **pl, int n_systems, const int *atom_off, const float *boxes,
                    const nb_config *cfg);

/* Free a pair list and its device buffers. Synchronises the device. NULL is a no-op. */
int nb_pairlist_destroy(nb_pairlist *pl);

/*
 * Pair search (§III-A, "pair list buffer" / "list range"): grid-sort atoms
 * into 8-atom clusters and build the outer cluster-pair list at radius
 * rlist.
 *   coords   device float[3*n_atoms], x,y,z per atom in original order;
 *            any real values (wrapped into the box here).
 *   box      HOST float[3], orthorhombic box edges; each > 2*rlist. Must be
 *            NULL for a batch (its boxes were fixed at nb_batch_create).
 *   rlist    list radius (nm), > 0.
 *   excl_off device int[n_atoms+1], excl_idx device int[excl_off[n]]:
 *            symmetric exclusion lists in original atom indices (both
 *            directions listed; self need not be). Both NULL = none.
 * The list keeps each cluster pair (ci <= cj) under each periodic shift
 * that brings it within rlist at most once, with a 64-bit mask of atom
 * pairs that are real, not excluded and not duplicated. Mask bit a*8+b is
 * atom a of ci with atom b of cj. A cluster pair can appear under two
 * shifts when rlist is close to half a box edge; an atom pair still has at
 * most one image within rlist (every edge exceeds 2*rlist).
 * After the search the forces use the outer list until nb_prune runs.
 * Device errors: NB_DEV_LIST_OVERFLOW, NB_DEV_COLUMN_OVERFLOW,
 * NB_DEV_NONFINITE, NB_DEV_EXCL_OVERFLOW.
 */
int nb_search(nb_pairlist *pl, const float *coords, const float *box, float rlist,
              const int *excl_off, const int *excl_idx, void *stream);

/*
 * Rolling prune (§III-A, "Prune-only kernel"): from the outer list keep the
 * cluster pairs with at least one masked-in atom pair closer than r_inner
 * at the given coordinates, and store per-atom-pair in-range masks. The
 * forces then use this inner list until the next nb_prune or nb_search.
 *   coords device float[3*n_atoms] (current frame), r_inner in (0, rlist].
 * Errors: NB_ERR_STATE before any search, NB_ERR_ARG for r_inner > rlist.
 * Device errors: NB_DEV_STALE_SEARCH if atoms moved more than
 * (rlist - r_inner)/2 since the search, NB_DEV_NONFINITE.
 */
int nb_prune(nb_pairlist *pl, const float *coords, float r_inner, void *stream);

/*
 * Forces and energies (§III-A, "NBNXM (short-range non-bonded forces)"),
 * FP32 arithmetic, FP64 energy reduction.
 *   coords   device float[3*n_atoms], current frame, original order.
 *   q        device float[n_atoms] charges (e).
 *   type     device int[n_atoms] LJ type in [0, ntype).
 *   ntype    1..32.
 *   ljparams device float[ntype*ntype*2] = (C6, C12) for type pair
 *            (ti, tj) at index 2*(ti*ntype + tj); symmetric.
 *   rc       cutoff (nm); <= r_inner if pruned, else <= rlist.
 *   beta     Ewald splitting parameter (nm^-1), 0 <= beta*rc <= 3.2.
 *   forces   device float[3*n_atoms], overwritten, original order.
 *   energies device double[2] = {E_LJ, E_C}, overwritten; may be NULL
 *            (forces only). For a batch: double[2*n_systems], one pair per
 *            system.
 * A pair counts iff its mask bit is set and r2 < fl(rc*rc) in FP32, with
 * d = (y_a - y_b) + S and r2 = fma(dz,dz,fma(dy,dy,dx*dx)); y is the image
 * of the current position nearest to the search-time wrapped position.
 * Errors: NB_ERR_STATE before any search; NB_ERR_ARG for bad ntype, rc, beta.
 * Device errors: NB_DEV_STALE_SEARCH / NB_DEV_STALE_PRUNE when the
 * displacement since the search / prune exceeds (rlist-rc)/2 / (r_inner-rc)/2
 * (minus 1e-5 nm), NB_DEV_NONFINITE, NB_DEV_BAD_TYPE.
 */
int nb_forces(nb_pairlist *pl, const float *coords, const float *q, const int *type, int ntype,
              const float *ljparams, float rc, float beta, float *forces, double *energies,
              void *stream);

/*
 * Adjoint of nb_forces (the "differentiation" form of the path; the paper
 * itself has no backward pass): given g = dL/dF for a scalar L of the
 * forces, the gradients of L with respect to positions, charges and the LJ
 * matrix, recomputing every pair term over the current list (nothing from
 * the forward call is stored).
 *   coords, q, type, ntype, ljparams, rc, beta: as for nb_forces;
 *            ntype <= NB_BACKWARD_MAX_TYPES.
 *   g        device float[3*n_atoms], dL/dF in original order.
 *   grad_x   device float[3*n_atoms], dL/dx (overwritten). With F = -dE/dx
 *            this is -H g, H the Hessian of E.
 *   grad_q   device float[n_atoms], dL/dq (overwritten).
 *   grad_lj  device double[ntype*ntype*2], dL/d(C6, C12) for the symmetric
 *            LJ matrix: each type pair's derivative is split evenly between
 *            entries (ti, tj) and (tj, ti) (overwritten).
 * Errors and device error bits as for nb_forces.
 */
#define NB_BACKWARD_MAX_TYPES 4
int nb_backward(nb_pairlist *pl, const float *coords, const float *q, const int *type, int ntype,
                const float *ljparams, float rc, float beta, const float *g, float *grad_x, float *grad_q,
                double *grad_lj, void *stream);

/*
 * Read the sticky device error word into *error_word (NB_DEV_* bits).
 * Synchronises the stream. clear != 0 resets the word after reading.
 */
int nb_status(nb_pairlist *pl, unsigned *error_word, int clear, void *stream);

/* Fill *out with list sizes, counters and radii. Synchronises the stream. */
int nb_pairlist_stats(nb_pairlist *pl, nb_stats *out, void *stream);

/* The displacement tracker (§III-A's rolling prune needs to know when the
   buffered list goes stale) and the error word, as of the last completed
   call in stream order. Squared displacements, as FP32. */
typedef struct {
    unsigned error_word;    /* sticky device error bits (NB_DEV_*) */
    float max_disp2_search; /* largest squared atom displacement since the search */
    float max_disp2_prune;  /* the same since the last prune */
} nb_tracker;

/*
 * Enqueue on `stream` a copy of the tracker into *out (12 bytes of host
 * memory that the caller owns and keeps valid until the stream has passed
 * the copy; page-locked memory keeps the copy asynchronous). Does not
 * synchronise: the values are there once the stream reaches this point,
 * e.g. after an event recorded right after this call. Lets a driver read
 * the tracker a few calls late without draining the stream.
 * Errors: NB_ERR_ARG for NULL arguments, NB_ERR_CUDA if the copy cannot be
 * enqueued.
 */
int nb_tracker_enqueue(nb_pairlist *pl, nb_tracker *out, void *stream);

/*
 * Copy a list to HOST arrays (for tests and inspection). Synchronises.
 *   which  NB_LIST_OUTER or NB_LIST_INNER.
 *   ci, cj, shift: int[cap]; mask: unsigned long long[cap]. shift is
 *   (sx+1)*9 + (sy+1)*3 + (sz+1) with S = (sx*Lx, sy*Ly, sz*Lz) added to
 *   (y_a - y_b), a in ci, b in cj.
 *   *n_out receives the entry count (also when it exceeds cap; then only
 *   cap entries are written and NB_ERR_CAPACITY is returned).
 *   perm: int[perm_cap] or NULL: atom of each cluster slot (slot = 8*c + a),
 *   -1 for padding; *n_slots receives 8*n_clusters.
 */
int nb_pairlist_export(nb_pairlist *pl, int which, int *ci, int *cj, int *shift,
                       unsigned long long *mask, size_t cap, size_t *n_out, int *perm,
                       size_t perm_cap, size_t *n_slots, void *stream);

/*
 * Copy the gathered tiles of the last prune to HOST arrays (tests and
 * inspection; synchronises). A prune also packs, for each half i-cluster
 * (half_id = 2*ci + h: rows 4h..4h+3 of cluster ci), the j atoms within
 * r_inner of any of its rows into tiles of 8: slots[8*k + p] is the cluster
 * slot of j atom p (low 27 bits) and its shift index (top 5 bits);
 * masks[k] bit a*8+p marks row a with atom p in range. After a prune
 * nb_forces and nb_backward compute over these tiles unless
 * NB_FLAG_CLUSTER_TILES is set.
 * half_id, masks: [cap]; slots: [8*cap]. *n_out receives the tile count.
 */
int nb_pairlist_export_tiles(nb_pairlist *pl, int *half_id, int *slots, unsigned *masks, size_t cap,
                             size_t *n_out, void *stream);

/*
 * Timing hook (no counterpart in the paper; measurement only): every later
 * nb_forces call records the caller's CUDA events `start` right before and
 * `stop` right after its force kernel, on the call's stream, so that the
 * kernel alone can be timed with cudaEventElapsedTime. Both NULL disables.
 * The events are caller-owned (cudaEvent_t passed as void*).
 */
int nb_set_timing_events(nb_pairlist *pl, void *start, void *stop);

/*
 * Replace the pair list's NB_FLAG_* flags (set at creation through
 * nb_config.flags). Each flag takes effect at the next call that reads it:
 * NB_FLAG_COUNT_PAIRS and NB_FLAG_CLUSTER_TILES at nb_forces / nb_backward,
 * NB_FLAG_NO_LIST_SORT at nb_search / nb_prune. Used by the autotuner to
 * choose the tile form. Errors: NB_ERR_ARG for an unknown flag.
 */
int nb_set_flags(nb_pairlist *pl, unsigned flags);

/*
 * Local / non-local split (the domain-decomposition form of the kernel,
 * §III-A: local work runs while the halo coordinates are still arriving).
 * Atoms [0, n_home) are home atoms and [n_home, n) halo atoms; the default
 * n_home = n means no halo. A pair is local when both atoms are home and
 * non-local otherwise. Takes effect at the next nb_search; single-system
 * pair lists only. Reserves the second region of gathered tiles (the pair
 * list's tile buffers double), so call it before any graph capture.
 * Errors: NB_ERR_ARG (n_home outside [1, n], a batch), NB_ERR_NOMEM.
 */
int nb_set_home(nb_pairlist *pl, int n_home);

/* nb_forces_part parts */
#define NB_PART_ALL 0      /* every pair (= nb_forces) */
#define NB_PART_LOCAL 1    /* pairs of two home atoms */
#define NB_PART_NONLOCAL 2 /* pairs with a halo atom */

/*
 * One part of nb_forces. NB_PART_LOCAL reads the home atoms' coordinates,
 * charges and types, zeroes the force accumulators and energies[], and
 * computes the local pairs; it writes nothing to forces (which may be NULL).
 * NB_PART_NONLOCAL, issued after NB_PART_LOCAL on the same stream (or one
 * that waits for it), reads the halo atoms' inputs, computes the non-local
 * pairs, adds their energies to energies[] and writes the total forces of
 * all atoms to forces. Between the two calls the caller may update the halo
 * atoms' coordinates (e.g. the copy of a halo exchange on another stream):
 * the local part never reads them. Without a halo, NB_PART_LOCAL computes
 * every pair and NB_PART_NONLOCAL only writes the forces. Arguments and
 * errors as nb_forces; NB_ERR_ARG for an unknown part.
 */
int nb_forces_part(nb_pairlist *pl, int part, const float *coords, const float *q, const int *type, int ntype,
                   const float *ljparams, float rc, float beta, float *forces, double *energies, void *stream);

/* Coulomb flavours (nb_set_coulomb). The paper's benchmark systems come in
   Ewald ("PME") and reaction-field ("RF") flavours (§II). */
#define NB_COUL_EWALD 0 /* real-space Ewald: f qi qj erfc(beta r)/r (default) */
#define NB_COUL_RF 1    /* reaction field: f qi qj (1/r + k_rf r^2 - c_rf) */
/* nb_set_coulomb flags */
#define NB_COUL_SHIFT 0x1u     /* Ewald only: subtract f qi qj erfc(beta rc)/rc from each pair energy */
#define NB_COUL_EXCL_CORR 0x2u /* add the excluded pairs within rc: Ewald -f qi qj erf(beta r)/r,
                                  RF f qi qj (k_rf r^2 - c_rf), with their forces */

/*
 * Coulomb flavour of later nb_forces / nb_backward calls on this pair list
 * (the default is NB_COUL_EWALD with no flags).
 *   kind    NB_COUL_EWALD or NB_COUL_RF. For RF, beta in nb_forces is
 *           ignored; k_rf = (eps_rf - 1) / ((2 eps_rf + 1) rc^3) and
 *           c_rf = 1/rc + k_rf rc^2 (permittivity 1 inside the cutoff), so
 *           the pair energy is 0 at rc.
 *   eps_rf  reaction-field permittivity: 0 means infinity (k_rf = 1/(2 rc^3)),
 *           otherwise >= 1. Ignored for Ewald.
 *   flags   NB_COUL_SHIFT (Ewald only) | NB_COUL_EXCL_CORR. The correction
 *           covers the excluded pairs of the exclusion lists given to the
 *           last nb_search: a search made while NB_COUL_EXCL_CORR is set
 *           keeps them as its own slot pairs (up to 8 per atom; beyond that
 *           NB_DEV_EXCL_OVERFLOW), so set the flag before the search; a
 *           force or adjoint call with the flag on a list searched without
 *           it fails with NB_ERR_STATE. Excluded pairs carry no LJ. The self
 *           terms (i = i) are constants the caller adds.
 * Energies: the corrections are part of E_coul. Errors: NB_ERR_ARG for an
 * unknown kind or flag, eps_rf in (0, 1), or NB_COUL_SHIFT with RF.
 */
int nb_set_coulomb(nb_pairlist *pl, int kind, float eps_rf, unsigned flags);

/*
 * Launch shape of the force kernel for later nb_forces calls on this pair
 * list (measurement and tuning; no counterpart in the paper). The results do
 * not depend on it, only the speed: threads per block (128 or 256), list
 * entries staged in shared memory per warp at a time (8 or 16) and CTAs per
 * SM of the persistent grid (at most what fits; 0 = as many as fit). Zero
 * for threads or chunk restores the default: 128 threads for the kernel over
 * gathered tiles (after a prune), 256 threads and chunks of 16 for the 8 x 8
 * cluster-pair kernel.
 */
int nb_set_force_shape(nb_pairlist *pl, int threads, int chunk, int blocks_per_sm);

/*
 * Smooth particle-mesh Ewald: charge spreading and force gathering.
 *
 * §III-A (Fig. 2 and the kernel list after it) names PME as the next
 * rate-limiting GPU work after the short-range kernel; the paper prints no
 * formulas, and these calls follow the smooth PME of Essmann et al.
 * (J. Chem. Phys. 103, 8577, 1995) with cardinal B-splines of order 4 in an
 * orthorhombic box. The FFT solve between them (Q -> phi) is not part of
 * this library: phi is whatever mesh potential the caller supplies (in
 * smooth PME, the reciprocal-space kernel convolved with Q).
 *
 *   u_a      = K_a x_a / L_a, the scaled fractional coordinate (any image of
 *              x is accepted; u is taken modulo K_a)
 *   M(u)     = the cubic cardinal B-spline, nonzero on (0, 4)
 *   Q(k)     = sum_i q_i prod_a M(u_ia - k_a)            (k_a taken mod K_a)
 *   psi_i    = sum_k prod_a M(u_ia - k_a) phi(k)
 *   F_ia     = -q_i dpsi_i/dx_ia
 *            = -q_i (K_a / L_a) sum_k M'(u_ia - k_a) prod_{b != a} M(u_ib - k_b) phi(k)
 *   energy   = (1/2) sum_i q_i psi_i   (= (1/2) sum_k Q(k) phi(k))
 *
 * Mesh layout: float[K0 * K1 * K2], index (k0 * K1 + k1) * K2 + k2 (the z
 * index fastest), device memory owned by the caller. Atoms in the caller's
 * order: coords float[3 n_atoms], q float[n_atoms], device. box is a HOST
 * float[3] (edges > 0). order must be 4 and each K_a in [4, 4096], else
 * NB_ERR_ARG; n_atoms = 0 is allowed. Arithmetic is FP32 with the scaled
 * coordinates formed as a two-float product (fractional parts exact to
 * about 2^-24 at any K); mesh values are summed with FP32 atomics, so their
 * last bits depend on the order the atoms land in. Non-finite coordinates
 * give NaN in the mesh or the forces, never an access outside the mesh.
 * Both calls are queued on stream and do not synchronise.
 */
/* grid (DEVICE float[K0*K1*K2]) is overwritten with Q. */
int nb_pme_spread(int n_atoms, const float *coords, const float *q, const float *box, int K0, int K1, int K2,
                  int order, float *grid, void *stream);
/* phi: DEVICE float[K0*K1*K2]. forces: DEVICE float[3 n_atoms], overwritten
 * (accumulate = 0) or added to (accumulate != 0). energy: DEVICE double[1]
 * or NULL; overwritten with (1/2) sum_i q_i psi_i, summed in FP64. */
int nb_pme_gather(int n_atoms, const float *coords, const float *q, const float *box, int K0, int K1, int K2,
                  int order, const float *phi, float *forces, int accumulate, double *energy, void *stream);

/*
 * FP32 throughput probe (measurement only; no counterpart in the paper).
 * The force kernel is bound by FP32 arithmetic, and this call measures the
 * rate its roofline divides by: a grid of blocks_per_sm (1..8) blocks of
 * 256 threads per SM, each thread running 8 independent fused
 * multiply-add chains for iters x 16 steps, as scalar FFMA (packed = 0) or
 * as two-wide FFMA2 (packed != 0, two fused multiply-adds per instruction).
 *
 *   out      DEVICE float[out_len], caller-owned; each thread writes its
 *            chains' sum (so nothing is optimised away). out_len must be at
 *            least SMs x blocks_per_sm x 256, else NB_ERR_ARG.
 *   flops    HOST double*: receives the launch's FP32 operations, counting
 *            a fused multiply-add as 2.
 *
 * The launch is queued on stream and not waited for: time it with events
 * recorded around the call. Returns NB_ERR_ARG for bad arguments and
 * NB_ERR_CUDA if the launch fails.
 */
int nb_fp32_peak_probe(int packed, int blocks_per_sm, int iters, float *out, size_t out_len, double *flops,
                       void *stream);

/*
 * Search and forces without any device allocation (no counterpart in the
 * paper; it exists for callers that cannot allocate device memory).
 *
 * Some callers cannot call cudaMalloc: a plug-in inside a host program that
 * owns every device allocation itself, or a real-time loop that must not
 * enter the allocator once it runs (cudaMalloc may synchronise the device
 * and take unbounded time). For them this entry point runs the same kernels
 * as nb_search + nb_forces (outer list at rlist = rc, no prune) with all
 * scratch memory (cluster grid, pair list, sorted coordinates, force
 * accumulators) in one statically allocated device array of
 * NB_NOALLOC_SCRATCH_BYTES bytes. Every GPU that loads libnb.so holds that
 * array until the process exits. The call allocates nothing: it makes no
 * cudaMalloc or cudaFree call and uses no allocating library routine.
 *
 *   n_atoms  1..NB_NOALLOC_MAX_ATOMS; larger systems return NB_ERR_CAPACITY
 *            (use nb_pairlist_create for them).
 *   coords, q, type, ljparams, excl_off, excl_idx, forces, energies:
 *            as for nb_search / nb_forces (device pointers, caller-owned).
 *   box      HOST float[3], each edge > 2*rc.
 *   rc, beta as for nb_forces (beta*rc <= 3.2).
 *   error_word  HOST unsigned* or NULL: if given, the call synchronises the
 *            stream and stores the device error word (NB_DEV_* bits) of
 *            this call; if NULL the call does not synchronise, and the errors
 *            the kernels find (a list overflow, non-finite coordinates, an LJ
 *            type out of range, too many exclusions in a cluster) are lost:
 *            there is no pair list to ask with nb_status, and the next call
 *            clears the word. Trust the results only when error_word is given
 *            and comes back 0.
 *
 * The pair list has room for NB_NOALLOC_MAX_ATOMS^2 / 64 entries (one per
 * cluster pair of a full half list, twice over), enough for a water-density
 * box at the largest cutoff the call accepts (rc just below half the
 * shortest box edge). A list that still overflows sets NB_DEV_LIST_OVERFLOW
 * in the error word and its forces are incomplete.
 *
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current); make that first call
 * before any stream capture. Every call shares the one array and each call
 * resets the parts that must start at zero; calls whose work overlaps on the
 * GPU (different streams or threads without ordering between them) race on
 * it and give wrong results.
 */
#define NB_NOALLOC_MAX_ATOMS 4096
#define NB_NOALLOC_SCRATCH_BYTES 5074432
int nb_forces_noalloc(int n_atoms, const float *coords, const float *box, const float *q, const int *type,
                      int ntype, const float *ljparams, float rc, float beta, const int *excl_off,
                      const int *excl_idx, float *forces, double *energies, unsigned *error_word,
                      void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NB_H */
