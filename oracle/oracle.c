/*
 * Plain CPU oracle for the short-range nonbonded path.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library. The product path never links,
 * loads or calls it, and it shares no code, header or constant with the
 * CUDA library.
 *
 * What it computes (the plain definition that the cluster-pair method of
 * §III-A, "NBNXM", reaches exactly up to rounding):
 *
 *   E_LJ = sum_{i<j, (i,j) not excluded, r_ij < rc}
 *            C12_ij / r^12 - C6_ij / r^6 - (C12_ij / rc^12 - C6_ij / rc^6)
 *   E_C  = f * sum_{i<j, not excluded, r_ij < rc} q_i q_j erfc(beta r) / r
 *   F_i  = -dE/dx_i
 *
 * with f = 138.935458 kJ mol^-1 nm e^-2, r_ij the minimum-image distance in
 * an orthorhombic box, and the cutoff test r < rc (strict). Everything is
 * FP64 with libm erfc/exp. The paper gives no formulas for the kernel
 * (§III-A names it "short-range non-bonded forces" with Ewald-type and
 * Lennard-Jones flavours); this is textbook LJ + Ewald real-space physics.
 *
 * oracle_energy_forces_coul / oracle_force_vjp_coul (end of this file) add
 * the reaction-field flavour, the Ewald potential shift and the
 * excluded-pair correction. oracle_energy_f32 (the end of this file) gives
 * the same energies at the distances the FP32 contract fixes.
 *
 * Pins (tests, CPU only): Coulomb's law at beta = 0, tabulated erfc values,
 * the LJ force zero at 2^(1/6) sigma and energy zero at sigma, continuity at
 * rc, sum of forces = 0, translation and permutation invariance, length
 * scaling laws, F = -dE/dx by central differences, O(N^2) == cell list, and
 * brute-force pair sets on tiny inputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_COULOMB_F 138.935458

static int oracle_nthreads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int oracle_tid(void) {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

int oracle_threads(void) { return oracle_nthreads(); }

/* Is j in the exclusion list of i? Self is always excluded. */
static int is_excluded(int i, int j, const int *excl_off, const int *excl_idx) {
    if (i == j) return 1;
    if (!excl_off) return 0;
    for (int k = excl_off[i]; k < excl_off[i + 1]; ++k)
        if (excl_idx[k] == j) return 1;
    return 0;
}

/* Minimum-image displacement x_i - x_j in FP64: d -= L * rint(d / L). */
static void min_image(const double *xi, const double *xj, const double *box, double *d) {
    for (int k = 0; k < 3; ++k) {
        double v = xi[k] - xj[k];
        v -= box[k] * rint(v / box[k]);
        d[k] = v;
    }
}

/*
 * One pair's contribution. Returns the pair energies and the scalar s such
 * that F_i += s * d and F_j -= s * d, with
 *   s = f q_i q_j [erfc(beta r)/r + 2 beta/sqrt(pi) exp(-beta^2 r^2)] / r^2
 *       + 12 C12 / r^14 - 6 C6 / r^8,
 * which is -(1/r) dE/dr for the pair energy above.
 */
static void pair_terms(double r2, double qi, double qj, double c6, double c12, double rc,
                       double beta, double *elj, double *ec, double *s) {
    double r = sqrt(r2);
    double rinv2 = 1.0 / r2;
    double rinv6 = rinv2 * rinv2 * rinv2;
    double rc6 = pow(rc, -6.0), rc12 = rc6 * rc6;
    *elj = c12 * rinv6 * rinv6 - c6 * rinv6 - (c12 * rc12 - c6 * rc6);
    double qq = ORACLE_COULOMB_F * qi * qj;
    double erfc_r = erfc(beta * r) / r;
    *ec = qq * erfc_r;
    double sc = qq * (erfc_r + 2.0 * beta / sqrt(M_PI) * exp(-beta * beta * r2)) * rinv2;
    double slj = (12.0 * c12 * rinv6 * rinv6 - 6.0 * c6 * rinv6) * rinv2;
    *s = sc + slj;
}

/* Cell grid for the cell-list path: nc[k] = floor(L_k / rc) cells per axis. */
static int cell_grid(const double *box, double rc, int *nc) {
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(box[k] / rc);
        if (nc[k] < 3) return 0; /* too few cells for a 27-cell stencil without repeats */
    }
    return 1;
}

static int cell_of(const double *x, const double *box, const int *nc) {
    int c[3];
    for (int k = 0; k < 3; ++k) {
        double w = x[k] - box[k] * floor(x[k] / box[k]);
        int ck = (int)floor(w / box[k] * nc[k]);
        if (ck < 0) ck = 0;
        if (ck >= nc[k]) ck = nc[k] - 1;
        c[k] = ck;
    }
    return (c[0] * nc[1] + c[1]) * nc[2] + c[2];
}

/* Counting sort of atoms by cell: cell_start[ncell + 1], cell_atoms[n]. */
static void build_cells(int n, const double *x, const double *box, const int *nc,
                        int *cell_start, int *cell_atoms, int *atom_cell) {
    int ncell = nc[0] * nc[1] * nc[2];
    memset(cell_start, 0, sizeof(int) * (size_t)(ncell + 1));
    for (int i = 0; i < n; ++i) {
        atom_cell[i] = cell_of(x + 3 * i, box, nc);
        cell_start[atom_cell[i] + 1]++;
    }
    for (int c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    int *fill = (int *)malloc(sizeof(int) * (size_t)ncell);
    memcpy(fill, cell_start, sizeof(int) * (size_t)ncell);
    for (int i = 0; i < n; ++i) cell_atoms[fill[atom_cell[i]]++] = i;
    free(fill);
}

/* The 27 neighbour cells of cell c (with periodic wrap). */
static void neighbour_cells(int c, const int *nc, int *out) {
    int cz = c % nc[2], cy = (c / nc[2]) % nc[1], cx = c / (nc[1] * nc[2]);
    int m = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int x = (cx + dx + nc[0]) % nc[0], y = (cy + dy + nc[1]) % nc[1],
                    z = (cz + dz + nc[2]) % nc[2];
                out[m++] = (x * nc[1] + y) * nc[2] + z;
            }
}

/*
 * Energies and forces in FP64.
 *   x[3n], q[n], type[n], lj[ntype*ntype*2] = (C6, C12) per type pair,
 *   box[3], excl CSR (may be NULL), method 0 = auto, 1 = O(N^2), 2 = cell list.
 * Outputs: F[3n] (overwritten), E[2] = {E_LJ, E_C}, *npairs = pairs counted,
 * Eabs[2] (may be NULL) = sums of the absolute pair energies |e_LJ|, |e_C|:
 * the scale that FP32 rounding errors of a pair sum are proportional to.
 * Returns 0, or -1 if rc >= L/2 on some axis, -2 if the cell list was asked
 * for but the box has fewer than 3 cells per axis.
 */
int oracle_energy_forces(int n, const double *x, const double *q, const int *type, int ntype,
                         const double *lj, const double *box, double rc, double beta,
                         const int *excl_off, const int *excl_idx, int method, double *F,
                         double *E, long long *npairs, double *Eabs) {
    for (int k = 0; k < 3; ++k)
        if (!(rc < 0.5 * box[k])) return -1;
    int nc[3];
    int have_cells = cell_grid(box, rc, nc);
    if (method == 2 && !have_cells) return -2;
    int use_cells = (method == 2) || (method == 0 && have_cells && n > 4096);

    int nt = oracle_nthreads();
    double *Ft = (double *)calloc((size_t)nt * 3 * (size_t)n, sizeof(double));
    double *Elj = (double *)calloc((size_t)nt, sizeof(double));
    double *Ec = (double *)calloc((size_t)nt, sizeof(double));
    long long *Np = (long long *)calloc((size_t)nt, sizeof(long long));
    double *Alj = (double *)calloc((size_t)nt, sizeof(double));
    double *Ac = (double *)calloc((size_t)nt, sizeof(double));
    double rc2 = rc * rc;

    int *cell_start = NULL, *cell_atoms = NULL, *atom_cell = NULL;
    if (use_cells) {
        int ncell = nc[0] * nc[1] * nc[2];
        cell_start = (int *)malloc(sizeof(int) * (size_t)(ncell + 1));
        cell_atoms = (int *)malloc(sizeof(int) * (size_t)n);
        atom_cell = (int *)malloc(sizeof(int) * (size_t)n);
        build_cells(n, x, box, nc, cell_start, cell_atoms, atom_cell);
    }

#pragma omp parallel
    {
        int tid = oracle_tid();
        double *Fl = Ft + (size_t)tid * 3 * (size_t)n;
        double elj_sum = 0.0, ec_sum = 0.0, alj_sum = 0.0, ac_sum = 0.0;
        long long np = 0;
        int nb[27];
#pragma omp for schedule(static)
        for (int i = 0; i < n; ++i) {
            int ncand_cells = use_cells ? 27 : 1;
            if (use_cells) neighbour_cells(atom_cell[i], nc, nb);
            for (int cc = 0; cc < ncand_cells; ++cc) {
                int j0, j1;
                if (use_cells) {
                    j0 = cell_start[nb[cc]];
                    j1 = cell_start[nb[cc] + 1];
                } else {
                    j0 = i + 1;
                    j1 = n;
                }
                for (int jj = j0; jj < j1; ++jj) {
                    int j = use_cells ? cell_atoms[jj] : jj;
                    if (j <= i) continue;
                    double d[3];
                    min_image(x + 3 * i, x + 3 * j, box, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (!(r2 < rc2)) continue;
                    if (is_excluded(i, j, excl_off, excl_idx)) continue;
                    const double *p = lj + 2 * ((size_t)type[i] * ntype + type[j]);
                    double elj, ec, s;
                    pair_terms(r2, q[i], q[j], p[0], p[1], rc, beta, &elj, &ec, &s);
                    elj_sum += elj;
                    ec_sum += ec;
                    alj_sum += fabs(elj);
                    ac_sum += fabs(ec);
                    np++;
                    for (int k = 0; k < 3; ++k) {
                        Fl[3 * i + k] += s * d[k];
                        Fl[3 * j + k] -= s * d[k];
                    }
                }
            }
        }
        Elj[tid] = elj_sum;
        Ec[tid] = ec_sum;
        Np[tid] = np;
        Alj[tid] = alj_sum;
        Ac[tid] = ac_sum;
    }
    /* fixed-order reduction: deterministic for a given thread count */
    for (size_t k = 0; k < 3 * (size_t)n; ++k) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += Ft[(size_t)t * 3 * (size_t)n + k];
        F[k] = s;
    }
    double el = 0.0, ecs = 0.0;
    long long npt = 0;
    for (int t = 0; t < nt; ++t) {
        el += Elj[t];
        ecs += Ec[t];
        npt += Np[t];
    }
    E[0] = el;
    E[1] = ecs;
    if (npairs) *npairs = npt;
    if (Eabs) {
        double a0 = 0.0, a1 = 0.0;
        for (int t = 0; t < nt; ++t) {
            a0 += Alj[t];
            a1 += Ac[t];
        }
        Eabs[0] = a0;
        Eabs[1] = a1;
    }
    free(Alj);
    free(Ac);
    free(Ft);
    free(Elj);
    free(Ec);
    free(Np);
    free(cell_start);
    free(cell_atoms);
    free(atom_cell);
    return 0;
}

/*
 * Forces on a subset of atoms, each summed over all its partners (no Newton's
 * third law), FP64. Used to check sampled atoms of systems too large to
 * compare in full. F_sub[3m]. Same return codes as oracle_energy_forces.
 */
int oracle_forces_subset(int n, const double *x, const double *q, const int *type, int ntype,
                         const double *lj, const double *box, double rc, double beta,
                         const int *excl_off, const int *excl_idx, int m, const int *atoms,
                         double *F_sub) {
    for (int k = 0; k < 3; ++k)
        if (!(rc < 0.5 * box[k])) return -1;
    int nc[3];
    int use_cells = cell_grid(box, rc, nc);
    int *cell_start = NULL, *cell_atoms = NULL, *atom_cell = NULL;
    if (use_cells) {
        int ncell = nc[0] * nc[1] * nc[2];
        cell_start = (int *)malloc(sizeof(int) * (size_t)(ncell + 1));
        cell_atoms = (int *)malloc(sizeof(int) * (size_t)n);
        atom_cell = (int *)malloc(sizeof(int) * (size_t)n);
        build_cells(n, x, box, nc, cell_start, cell_atoms, atom_cell);
    }
    double rc2 = rc * rc;
#pragma omp parallel for schedule(static)
    for (int t = 0; t < m; ++t) {
        int i = atoms[t];
        double f[3] = {0.0, 0.0, 0.0};
        int nb[27];
        int ncc = use_cells ? 27 : 1;
        if (use_cells) neighbour_cells(atom_cell[i], nc, nb);
        for (int cc = 0; cc < ncc; ++cc) {
            int j0 = use_cells ? cell_start[nb[cc]] : 0;
            int j1 = use_cells ? cell_start[nb[cc] + 1] : n;
            for (int jj = j0; jj < j1; ++jj) {
                int j = use_cells ? cell_atoms[jj] : jj;
                if (j == i) continue;
                double d[3];
                min_image(x + 3 * i, x + 3 * j, box, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < rc2)) continue;
                if (is_excluded(i, j, excl_off, excl_idx)) continue;
                const double *p = lj + 2 * ((size_t)type[i] * ntype + type[j]);
                double elj, ec, s;
                pair_terms(r2, q[i], q[j], p[0], p[1], rc, beta, &elj, &ec, &s);
                for (int k = 0; k < 3; ++k) f[k] += s * d[k];
            }
        }
        for (int k = 0; k < 3; ++k) F_sub[3 * t + k] = f[k];
    }
    free(cell_start);
    free(cell_atoms);
    free(atom_cell);
    return 0;
}

/*
 * Brute-force FP64 set of non-excluded pairs (i < j) with minimum-image
 * r < r_cut. O(N^2). Writes up to cap pairs to pi/pj and the total count to
 * *count. Returns 0, or 1 if cap was too small.
 */
int oracle_pairs_f64(int n, const double *x, const double *box, double r_cut,
                     const int *excl_off, const int *excl_idx, int *pi, int *pj, long long cap,
                     long long *count) {
    long long c = 0;
    double r2c = r_cut * r_cut;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double d[3];
            min_image(x + 3 * i, x + 3 * j, box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < r2c) || is_excluded(i, j, excl_off, excl_idx)) continue;
            if (c < cap) {
                pi[c] = i;
                pj[c] = j;
            }
            c++;
        }
    *count = c;
    return c > cap ? 1 : 0;
}

/* ------------------------------------------------------------------------
 * FP32 pair-set contract.
 *
 * The cluster-pair list is exact if the set of atom pairs the force kernel
 * counts equals the set of pairs within rc, where "within rc" is decided in
 * FP32 on the same FP32 coordinates. These functions state that decision as
 * plain C (compile with -ffp-contract=off):
 *
 *   wrap:   w = x - L*floor(x/L); if (w < 0) w += L; if (w >= L) w -= L;
 *           if (!(w >= 0 && w < L)) w = 0                (search frame x0)
 *   image:  k = rint((x - w0)/L); y = x - k*L            (current frame x)
 *   d:      d = (y_a - y_b) + S, S = s*L with s in {-1, 0, 1} per axis
 *   r2:     r2 = fmaf(dz, dz, fmaf(dy, dy, dx*dx))
 *   test:   r2 < rc*rc  (both FP32, rc*rc rounded once)
 *
 * d is antisymmetric in (a, b) with S -> -S, so the decision does not depend
 * on which atom sits in the i-cluster.
 * ------------------------------------------------------------------------ */
static float wrap32(float x, float L) {
    float w = x - L * floorf(x / L);
    if (w < 0.0f) w += L;
    if (w >= L) w -= L;
    if (!(w >= 0.0f && w < L)) w = 0.0f;
    return w;
}

static float image32(float x, float w0, float L) {
    float k = rintf((x - w0) / L);
    return x - k * L;
}

static float r2_32(float dx, float dy, float dz) {
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

/* FP32 positions used by the contract: y = image(x, wrap(x0)). y[3n] out. */
void oracle_image_f32(int n, const float *x0, const float *x, const float *box, float *y) {
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) y[3 * i + k] = image32(x[3 * i + k], wrap32(x0[3 * i + k], box[k]), box[k]);
}

/*
 * Set of non-excluded pairs (i < j) that are within rc under the FP32
 * contract above. Candidates come from an FP64 cell search with a 1e-3 nm
 * margin, far above FP32 rounding, so the margin never decides membership.
 * pi/pj may be NULL (count only). Returns 0; 1 if cap was too small; -1 if
 * rc >= L/2 (images would not be unique); -3 if some pair is within rc
 * for two different shifts.
 */
int oracle_pairs_f32(int n, const float *x0, const float *x, const float *box, float rc,
                     const int *excl_off, const int *excl_idx, int *pi, int *pj, long long cap,
                     long long *count) {
    for (int k = 0; k < 3; ++k)
        if (!(rc < 0.5f * box[k])) return -1;
    float *y = (float *)malloc(sizeof(float) * 3 * (size_t)n);
    oracle_image_f32(n, x0, x, box, y);
    double *yd = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    for (size_t k = 0; k < 3 * (size_t)n; ++k) yd[k] = (double)y[k];
    double bd[3] = {box[0], box[1], box[2]};
    double rsearch = (double)rc + 1e-3;
    int nc[3];
    int use_cells = 1;
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(bd[k] / rsearch);
        if (nc[k] < 3) use_cells = 0;
    }
    int *cell_start = NULL, *cell_atoms = NULL, *atom_cell = NULL;
    if (use_cells) {
        int ncell = nc[0] * nc[1] * nc[2];
        cell_start = (int *)malloc(sizeof(int) * (size_t)(ncell + 1));
        cell_atoms = (int *)malloc(sizeof(int) * (size_t)n);
        atom_cell = (int *)malloc(sizeof(int) * (size_t)n);
        build_cells(n, yd, bd, nc, cell_start, cell_atoms, atom_cell);
    }
    float rc2 = rc * rc;
    double rs2 = rsearch * rsearch;
    long long c = 0;
    int status = 0;
    int nb[27];
    for (int i = 0; i < n; ++i) {
        int ncc = use_cells ? 27 : 1;
        if (use_cells) neighbour_cells(atom_cell[i], nc, nb);
        for (int cc = 0; cc < ncc; ++cc) {
            int j0 = use_cells ? cell_start[nb[cc]] : i + 1;
            int j1 = use_cells ? cell_start[nb[cc] + 1] : n;
            for (int jj = j0; jj < j1; ++jj) {
                int j = use_cells ? cell_atoms[jj] : jj;
                if (j <= i) continue;
                double dd[3];
                min_image(yd + 3 * i, yd + 3 * j, bd, dd);
                if (!(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2] < rs2)) continue;
                if (is_excluded(i, j, excl_off, excl_idx)) continue;
                int hits = 0;
                float u[3];
                for (int k = 0; k < 3; ++k) u[k] = y[3 * i + k] - y[3 * j + k];
                for (int sx = -1; sx <= 1; ++sx)
                    for (int sy = -1; sy <= 1; ++sy)
                        for (int sz = -1; sz <= 1; ++sz) {
                            float dx = u[0] + (float)sx * box[0];
                            float dy = u[1] + (float)sy * box[1];
                            float dz = u[2] + (float)sz * box[2];
                            if (r2_32(dx, dy, dz) < rc2) hits++;
                        }
                if (hits > 1) status = -3;
                if (hits >= 1) {
                    if (pi && c < cap) {
                        pi[c] = i;
                        pj[c] = j;
                    }
                    c++;
                }
            }
        }
    }
    *count = c;
    free(y);
    free(yd);
    free(cell_start);
    free(cell_atoms);
    free(atom_cell);
    if (status) return status;
    return (pi && c > cap) ? 1 : 0;
}

/* ------------------------------------------------------------------------
 * Adjoint of the forces (vector-Jacobian product), FP64.
 *
 * Given g = dL/dF for some scalar L(F) (e.g. a force-matching loss), returns
 *   gx = dL/dx = sum_i g_i . dF_i/dx,   gq = dL/dq,   glj = dL/d(C6, C12).
 * Per pair (i, j) with d = x_i - x_j, F_i += s d, F_j -= s d, so the pair's
 * part of g.F is s(r) (u . d) with u = g_i - g_j, and
 *   d/dx_i [s (u.d)] = s u + (s'/r)(u.d) d           (= -d/dx_j)
 *   d/dq_i = f q_j B (u.d), d/dq_j = f q_i B (u.d),  B = [erfc(br)/r + c e]/r^2
 *   d/dC6 = -6 r^-8 (u.d),  d/dC12 = 12 r^-14 (u.d)
 * with c = 2b/sqrt(pi), e = exp(-b^2 r^2) and
 *   s'/r = -3 s_C / r^2 - 2 f q_i q_j c b^2 e / r^2 - 168 C12 r^-16 + 48 C6 r^-10.
 * The LJ matrix is one symmetric parameter set: the derivative for a type
 * pair {a, b} is split evenly between entries (a, b) and (b, a), so that
 * glj is symmetric and a symmetric perturbation of both entries changes L
 * by (glj[a][b] + glj[b][a]) times the step.
 * gx[3n], gq[n], glj[ntype*ntype*2] are overwritten. Same return codes as
 * oracle_energy_forces. Pinned by finite differences of g.F and by the
 * symmetry of the Hessian (tests/test_oracle_adjoint.py).
 * ------------------------------------------------------------------------ */
int oracle_force_vjp(int n, const double *x, const double *q, const int *type, int ntype,
                     const double *lj, const double *box, double rc, double beta,
                     const int *excl_off, const int *excl_idx, const double *g, double *gx,
                     double *gq, double *glj) {
    for (int k = 0; k < 3; ++k)
        if (!(rc < 0.5 * box[k])) return -1;
    int nc[3];
    int use_cells = cell_grid(box, rc, nc) && n > 4096;
    int nt = oracle_nthreads();
    size_t nlj = (size_t)ntype * ntype * 2;
    double *gxt = (double *)calloc((size_t)nt * 3 * (size_t)n, sizeof(double));
    double *gqt = (double *)calloc((size_t)nt * (size_t)n, sizeof(double));
    double *gljt = (double *)calloc((size_t)nt * nlj, sizeof(double));
    int *cell_start = NULL, *cell_atoms = NULL, *atom_cell = NULL;
    if (use_cells) {
        int ncell = nc[0] * nc[1] * nc[2];
        cell_start = (int *)malloc(sizeof(int) * (size_t)(ncell + 1));
        cell_atoms = (int *)malloc(sizeof(int) * (size_t)n);
        atom_cell = (int *)malloc(sizeof(int) * (size_t)n);
        build_cells(n, x, box, nc, cell_start, cell_atoms, atom_cell);
    }
    const double rc2 = rc * rc;
    const double cb = 2.0 * beta / sqrt(M_PI);
#pragma omp parallel
    {
        int tid = oracle_tid();
        double *gxl = gxt + (size_t)tid * 3 * (size_t)n;
        double *gql = gqt + (size_t)tid * (size_t)n;
        double *gljl = gljt + (size_t)tid * nlj;
        int nb[27];
#pragma omp for schedule(static)
        for (int i = 0; i < n; ++i) {
            int ncc = use_cells ? 27 : 1;
            if (use_cells) neighbour_cells(atom_cell[i], nc, nb);
            for (int cc = 0; cc < ncc; ++cc) {
                int j0 = use_cells ? cell_start[nb[cc]] : i + 1;
                int j1 = use_cells ? cell_start[nb[cc] + 1] : n;
                for (int jj = j0; jj < j1; ++jj) {
                    int j = use_cells ? cell_atoms[jj] : jj;
                    if (j <= i) continue;
                    double d[3];
                    min_image(x + 3 * i, x + 3 * j, box, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (!(r2 < rc2)) continue;
                    if (is_excluded(i, j, excl_off, excl_idx)) continue;
                    const double *p = lj + 2 * ((size_t)type[i] * ntype + type[j]);
                    double c6 = p[0], c12 = p[1];
                    double r = sqrt(r2), rinv2 = 1.0 / r2, rinv6 = rinv2 * rinv2 * rinv2;
                    double K = ORACLE_COULOMB_F * q[i] * q[j];
                    double e = exp(-beta * beta * r2);
                    double A = erfc(beta * r) / r;
                    double B = (A + cb * e) * rinv2;
                    double sC = K * B;
                    double sLJ = (12.0 * c12 * rinv6 * rinv6 - 6.0 * c6 * rinv6) * rinv2;
                    double s = sC + sLJ;
                    double spr = -3.0 * sC * rinv2 - 2.0 * K * cb * beta * beta * e * rinv2 -
                                 168.0 * c12 * rinv6 * rinv6 * rinv2 * rinv2 + 48.0 * c6 * rinv6 * rinv2 * rinv2;
                    double u[3], ud = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        u[k] = g[3 * i + k] - g[3 * j + k];
                        ud += u[k] * d[k];
                    }
                    for (int k = 0; k < 3; ++k) {
                        double v = s * u[k] + spr * ud * d[k];
                        gxl[3 * i + k] += v;
                        gxl[3 * j + k] -= v;
                    }
                    gql[i] += ORACLE_COULOMB_F * q[j] * B * ud;
                    gql[j] += ORACLE_COULOMB_F * q[i] * B * ud;
                    double d6 = -6.0 * rinv6 * rinv2 * ud, d12 = 12.0 * rinv6 * rinv6 * rinv2 * ud;
                    size_t ab = 2 * ((size_t)type[i] * ntype + type[j]);
                    size_t ba = 2 * ((size_t)type[j] * ntype + type[i]);
                    gljl[ab] += 0.5 * d6;
                    gljl[ab + 1] += 0.5 * d12;
                    gljl[ba] += 0.5 * d6;
                    gljl[ba + 1] += 0.5 * d12;
                }
            }
        }
    }
    for (size_t k = 0; k < 3 * (size_t)n; ++k) {
        double v = 0.0;
        for (int t = 0; t < nt; ++t) v += gxt[(size_t)t * 3 * (size_t)n + k];
        gx[k] = v;
    }
    for (size_t k = 0; k < (size_t)n; ++k) {
        double v = 0.0;
        for (int t = 0; t < nt; ++t) v += gqt[(size_t)t * (size_t)n + k];
        gq[k] = v;
    }
    for (size_t k = 0; k < nlj; ++k) {
        double v = 0.0;
        for (int t = 0; t < nt; ++t) v += gljt[(size_t)t * nlj + k];
        glj[k] = v;
    }
    free(gxt);
    free(gqt);
    free(gljt);
    free(cell_start);
    free(cell_atoms);
    free(atom_cell);
    return 0;
}

/* ------------------------------------------------------------------------
 * Coulomb options: the reaction-field flavour, the Ewald potential shift
 * and the exclusion correction (the paper's benchmark systems come in
 * Ewald "PME" and reaction-field "RF" flavours, §II; GROMACS's NBNXM kernels
 * have both). Per pair at distance r, per unit f q_i q_j, with
 *   E_C = f q_i q_j phi(r),  F_i += f q_i q_j B(r) d,  B = -(1/r) dphi/dr,
 *   D = (1/r) dB/dr (what the adjoint needs):
 *
 *   Ewald:            phi = erfc(beta r)/r - shift,
 *                     B = [erfc(beta r)/r + (2 beta/sqrt(pi)) exp(-beta^2 r^2)] / r^2,
 *                     D = [-3 B - 2 (2 beta/sqrt(pi)) beta^2 exp(-beta^2 r^2)] / r^2,
 *                     shift = erfc(beta rc)/rc with ORACLE_COUL_SHIFT, else 0;
 *   Ewald, excluded:  phi = -erf(beta r)/r (= erfc(beta r)/r - 1/r),
 *                     B = B_Ewald - 1/r^3, D = D_Ewald + 3/r^5;
 *   reaction field:   phi = 1/r + k_rf r^2 - c_rf,  B = 1/r^3 - 2 k_rf,  D = -3/r^5;
 *   RF, excluded:     phi = k_rf r^2 - c_rf,  B = -2 k_rf,  D = 0;
 *
 * with k_rf = (eps_rf - 1) / ((2 eps_rf + 1) rc^3), eps_rf = 0 meaning
 * infinity (k_rf = 1 / (2 rc^3)), relative permittivity 1 inside the
 * cutoff, and c_rf = 1/rc + k_rf rc^2 (phi_RF(rc) = 0). Excluded pairs
 * (from the exclusion lists, r < rc) contribute only with
 * ORACLE_COUL_EXCL_CORR, and never LJ. The self terms (i = i) are
 * constants a caller adds; they are not here.
 * ------------------------------------------------------------------------ */

#define ORACLE_COUL_EWALD 0
#define ORACLE_COUL_RF 1
#define ORACLE_COUL_SHIFT 0x1
#define ORACLE_COUL_EXCL_CORR 0x2

static void rf_constants(double rc, double eps_rf, double *k_rf, double *c_rf) {
    if (eps_rf == 0.0)
        *k_rf = 1.0 / (2.0 * rc * rc * rc);
    else
        *k_rf = (eps_rf - 1.0) / ((2.0 * eps_rf + 1.0) * rc * rc * rc);
    *c_rf = 1.0 / rc + *k_rf * rc * rc;
}

static void coul_radial(int kind, int excluded, double r, double beta, double k_rf, double c_rf,
                        double shift, double *phi, double *B, double *D) {
    double r2 = r * r, rinv2 = 1.0 / r2;
    if (kind == ORACLE_COUL_RF) {
        if (excluded) {
            *phi = k_rf * r2 - c_rf;
            *B = -2.0 * k_rf;
            *D = 0.0;
        } else {
            *phi = 1.0 / r + k_rf * r2 - c_rf;
            *B = rinv2 / r - 2.0 * k_rf;
            *D = -3.0 * rinv2 * rinv2 / r;
        }
        return;
    }
    double cb = 2.0 * beta / sqrt(M_PI);
    double e = exp(-beta * beta * r2);
    double A = erfc(beta * r) / r;
    double Be = (A + cb * e) * rinv2;
    double De = (-3.0 * Be - 2.0 * cb * beta * beta * e) * rinv2;
    if (excluded) {
        *phi = -erf(beta * r) / r;
        *B = Be - rinv2 / r;
        *D = De + 3.0 * rinv2 * rinv2 / r;
    } else {
        *phi = A - shift;
        *B = Be;
        *D = De;
    }
}

/* Energies and forces with Coulomb options; E[0] = E_LJ, E[1] = E_C
   (including excluded-pair corrections), *npairs = non-excluded pairs
   within rc. O(N^2) over i < j (cell list when n > 4096 and the box allows). */
int oracle_energy_forces_coul(int n, const double *x, const double *q, const int *type, int ntype,
                              const double *lj, const double *box, double rc, double beta,
                              const int *excl_off, const int *excl_idx, int kind, double eps_rf,
                              int flags, double *F, double *E, long long *npairs) {
    for (int k = 0; k < 3; ++k)
        if (!(rc < 0.5 * box[k])) return -1;
    if (kind != ORACLE_COUL_EWALD && kind != ORACLE_COUL_RF) return -3;
    int nc[3];
    int use_cells = cell_grid(box, rc, nc) && n > 4096;
    double k_rf = 0.0, c_rf = 0.0;
    if (kind == ORACLE_COUL_RF) rf_constants(rc, eps_rf, &k_rf, &c_rf);
    double shift = (kind == ORACLE_COUL_EWALD && (flags & ORACLE_COUL_SHIFT)) ? erfc(beta * rc) / rc : 0.0;
    int corr = (flags & ORACLE_COUL_EXCL_CORR) != 0;
    double rc6 = pow(rc, -6.0), rc12 = rc6 * rc6;
    int nt = oracle_nthreads();
    double *Ft = (double *)calloc((size_t)nt * 3 * (size_t)n, sizeof(double));
    double *Elj = (double *)calloc((size_t)nt, sizeof(double));
    double *Ec = (double *)calloc((size_t)nt, sizeof(double));
    long long *Np = (long long *)calloc((size_t)nt, sizeof(long long));
    int *cell_start = NULL, *cell_atoms = NULL, *atom_cell = NULL;
    if (use_cells) {
        int ncell = nc[0] * nc[1] * nc[2];
        cell_start = (int *)malloc(sizeof(int) * (size_t)(ncell + 1));
        cell_atoms = (int *)malloc(sizeof(int) * (size_t)n);
        atom_cell = (int *)malloc(sizeof(int) * (size_t)n);
        build_cells(n, x, box, nc, cell_start, cell_atoms, atom_cell);
    }
    const double rc2 = rc * rc;
#pragma omp parallel
    {
        int tid = oracle_tid();
        double *Fl = Ft + (size_t)tid * 3 * (size_t)n;
        double elj_sum = 0.0, ec_sum = 0.0;
        long long np = 0;
        int nb[27];
#pragma omp for schedule(static)
        for (int i = 0; i < n; ++i) {
            int ncc = use_cells ? 27 : 1;
            if (use_cells) neighbour_cells(atom_cell[i], nc, nb);
            for (int cc = 0; cc < ncc; ++cc) {
                int j0 = use_cells ? cell_start[nb[cc]] : i + 1;
                int j1 = use_cells ? cell_start[nb[cc] + 1] : n;
                for (int jj = j0; jj < j1; ++jj) {
                    int j = use_cells ? cell_atoms[jj] : jj;
                    if (j <= i) continue;
                    double d[3];
                    min_image(x + 3 * i, x + 3 * j, box, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (!(r2 < rc2)) continue;
                    int excl = is_excluded(i, j, excl_off, excl_idx);
                    if (excl && !corr) continue;
                    double r = sqrt(r2), phi, B, D;
                    coul_radial(kind, excl, r, beta, k_rf, c_rf, shift, &phi, &B, &D);
                    double K = ORACLE_COULOMB_F * q[i] * q[j];
                    double s = K * B;
                    ec_sum += K * phi;
                    if (!excl) {
                        const double *p = lj + 2 * ((size_t)type[i] * ntype + type[j]);
                        double rinv2 = 1.0 / r2, rinv6 = rinv2 * rinv2 * rinv2;
                        elj_sum += p[1] * rinv6 * rinv6 - p[0] * rinv6 - (p[1] * rc12 - p[0] * rc6);
                        s += (12.0 * p[1] * rinv6 * rinv6 - 6.0 * p[0] * rinv6) * rinv2;
                        np++;
                    }
                    for (int k = 0; k < 3; ++k) {
                        Fl[3 * i + k] += s * d[k];
                        Fl[3 * j + k] -= s * d[k];
                    }
                }
            }
        }
        Elj[tid] = elj_sum;
        Ec[tid] = ec_sum;
        Np[tid] = np;
    }
    for (size_t k = 0; k < 3 * (size_t)n; ++k) {
        double v = 0.0;
        for (int t = 0; t < nt; ++t) v += Ft[(size_t)t * 3 * (size_t)n + k];
        F[k] = v;
    }
    double el = 0.0, ecs = 0.0;
    long long npt = 0;
    for (int t = 0; t < nt; ++t) {
        el += Elj[t];
        ecs += Ec[t];
        npt += Np[t];
    }
    E[0] = el;
    E[1] = ecs;
    if (npairs) *npairs = npt;
    free(Ft);
    free(Elj);
    free(Ec);
    free(Np);
    free(cell_start);
    free(cell_atoms);
    free(atom_cell);
    return 0;
}

/* Adjoint of oracle_energy_forces_coul for g = dL/dF: per pair with
   u = g_i - g_j and s = f q_i q_j B + s_LJ,
     dL/dx_i += s u + (s'/r)(u.d) d,  dL/dx_j -= the same,
     s'/r = f q_i q_j D + (48 C6 / r^10 - 168 C12 / r^16),
     dL/dq_i += f q_j B (u.d),  dL/dq_j += f q_i B (u.d),
     dL/dC6 += -6 (u.d) / r^8,  dL/dC12 += 12 (u.d) / r^14 (non-excluded pairs),
   the LJ gradient split evenly between (t_i, t_j) and (t_j, t_i). */
int oracle_force_vjp_coul(int n, const double *x, const double *q, const int *type, int ntype,
                          const double *lj, const double *box, double rc, double beta,
                          const int *excl_off, const int *excl_idx, int kind, double eps_rf, int flags,
                          const double *g, double *gx, double *gq, double *glj) {
    for (int k = 0; k < 3; ++k)
        if (!(rc < 0.5 * box[k])) return -1;
    if (kind != ORACLE_COUL_EWALD && kind != ORACLE_COUL_RF) return -3;
    double k_rf = 0.0, c_rf = 0.0;
    if (kind == ORACLE_COUL_RF) rf_constants(rc, eps_rf, &k_rf, &c_rf);
    int corr = (flags & ORACLE_COUL_EXCL_CORR) != 0;
    size_t nlj = (size_t)ntype * ntype * 2;
    memset(gx, 0, sizeof(double) * 3 * (size_t)n);
    memset(gq, 0, sizeof(double) * (size_t)n);
    memset(glj, 0, sizeof(double) * nlj);
    const double rc2 = rc * rc;
    /* plain O(N^2) double loop: the adjoint tests use small systems */
    for (int i = 0; i < n; ++i) {
        for (int j = i + 1; j < n; ++j) {
            double d[3];
            min_image(x + 3 * i, x + 3 * j, box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc2)) continue;
            int excl = is_excluded(i, j, excl_off, excl_idx);
            if (excl && !corr) continue;
            double r = sqrt(r2), phi, B, D;
            coul_radial(kind, excl, r, beta, k_rf, c_rf, 0.0, &phi, &B, &D);
            double K = ORACLE_COULOMB_F * q[i] * q[j];
            double s = K * B, spr = K * D;
            double rinv2 = 1.0 / r2, rinv6 = rinv2 * rinv2 * rinv2;
            const double *p = lj + 2 * ((size_t)type[i] * ntype + type[j]);
            if (!excl) {
                s += (12.0 * p[1] * rinv6 * rinv6 - 6.0 * p[0] * rinv6) * rinv2;
                spr += (48.0 * p[0] * rinv6 - 168.0 * p[1] * rinv6 * rinv6) * rinv2 * rinv2;
            }
            double u[3], ud = 0.0;
            for (int k = 0; k < 3; ++k) {
                u[k] = g[3 * i + k] - g[3 * j + k];
                ud += u[k] * d[k];
            }
            for (int k = 0; k < 3; ++k) {
                double v = s * u[k] + spr * ud * d[k];
                gx[3 * i + k] += v;
                gx[3 * j + k] -= v;
            }
            gq[i] += ORACLE_COULOMB_F * q[j] * B * ud;
            gq[j] += ORACLE_COULOMB_F * q[i] * B * ud;
            if (!excl) {
                double d6 = -6.0 * rinv6 * rinv2 * ud, d12 = 12.0 * rinv6 * rinv6 * rinv2 * ud;
                size_t ab = 2 * ((size_t)type[i] * ntype + type[j]);
                size_t ba = 2 * ((size_t)type[j] * ntype + type[i]);
                glj[ab] += 0.5 * d6;
                glj[ab + 1] += 0.5 * d12;
                glj[ba] += 0.5 * d6;
                glj[ba + 1] += 0.5 * d12;
            }
        }
    }
    return 0;
}

/* As oracle_energy_forces_coul, with the set of non-excluded pairs given
   explicitly (pairs[2k], pairs[2k+1], i < j, npairs of them) instead of
   decided by r < rc in FP64: a caller that decides the in/out question in
   another precision (the FP32 contract) passes that set here. Excluded
   pairs (ORACLE_COUL_EXCL_CORR) still come from the exclusion lists with
   r < rc. Everything else is FP64 as above. */
int oracle_energy_forces_coul_list(int n, const double *x, const double *q, const int *type, int ntype,
                                   const double *lj, const double *box, double rc, double beta,
                                   const int *excl_off, const int *excl_idx, int kind, double eps_rf,
                                   int flags, const long long *pairs, long long npairs, double *F,
                                   double *E) {
    if (kind != ORACLE_COUL_EWALD && kind != ORACLE_COUL_RF) return -3;
    double k_rf = 0.0, c_rf = 0.0;
    if (kind == ORACLE_COUL_RF) rf_constants(rc, eps_rf, &k_rf, &c_rf);
    double shift = (kind == ORACLE_COUL_EWALD && (flags & ORACLE_COUL_SHIFT)) ? erfc(beta * rc) / rc : 0.0;
    double rc6 = pow(rc, -6.0), rc12 = rc6 * rc6;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    double elj = 0.0, ec = 0.0;
    for (long long k = 0; k < npairs; ++k) {
        int i = (int)pairs[2 * k], j = (int)pairs[2 * k + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) return -4;
        double d[3];
        min_image(x + 3 * i, x + 3 * j, box, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double r = sqrt(r2), phi, B, D;
        coul_radial(kind, 0, r, beta, k_rf, c_rf, shift, &phi, &B, &D);
        double K = ORACLE_COULOMB_F * q[i] * q[j];
        const double *p = lj + 2 * ((size_t)type[i] * ntype + type[j]);
        double rinv2 = 1.0 / r2, rinv6 = rinv2 * rinv2 * rinv2;
        double s = K * B + (12.0 * p[1] * rinv6 * rinv6 - 6.0 * p[0] * rinv6) * rinv2;
        ec += K * phi;
        elj += p[1] * rinv6 * rinv6 - p[0] * rinv6 - (p[1] * rc12 - p[0] * rc6);
        for (int c = 0; c < 3; ++c) {
            F[3 * i + c] += s * d[c];
            F[3 * j + c] -= s * d[c];
        }
    }
    if ((flags & ORACLE_COUL_EXCL_CORR) && excl_off) {
        for (int i = 0; i < n; ++i) {
            for (int e = excl_off[i]; e < excl_off[i + 1]; ++e) {
                int j = excl_idx[e];
                if (j <= i || j >= n) continue;
                double d[3];
                min_image(x + 3 * i, x + 3 * j, box, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < rc * rc)) continue;
                double phi, B, D;
                coul_radial(kind, 1, sqrt(r2), beta, k_rf, c_rf, 0.0, &phi, &B, &D);
                double K = ORACLE_COULOMB_F * q[i] * q[j];
                ec += K * phi;
                for (int c = 0; c < 3; ++c) {
                    F[3 * i + c] += K * B * d[c];
                    F[3 * j + c] -= K * B * d[c];
                }
            }
        }
    }
    E[0] = elj;
    E[1] = ec;
    return 0;
}

/* ------------------------------------------------------------------------
 * Smooth particle-mesh Ewald: charge spreading and force gathering.
 *
 * The paper names PME the rate limiter after the short-range kernel
 * (§III-A, Fig. 2) and gives no formulas. This follows the smooth PME of
 * Essmann et al. (J. Chem. Phys. 103, 8577, 1995), orthorhombic box:
 *
 *   scaled fractional coordinate  u_a = K_a * (x_a / L_a wrapped into [0, 1))
 *   cardinal B-spline of order n  M_2(u) = 1 - |u - 1| on [0, 2], else 0;
 *                                  M_n(u) = u/(n-1) M_{n-1}(u)
 *                                         + (n-u)/(n-1) M_{n-1}(u-1)
 *                                  dM_n/du = M_{n-1}(u) - M_{n-1}(u-1)
 *   spread   Q(k) = sum_i q_i sum_{images} prod_a M_n(u_ia - k_a - m_a K_a)
 *   gather   psi_i = sum_k prod_a M_n(u_ia - k_a) phi(k)   (interpolated potential)
 *            F_ia  = -q_i dpsi_i/dx_ia
 *                  = -q_i (K_a/L_a) sum_k M_n'(u_ia - k_a) prod_{b!=a} M_n(u_ib - k_b) phi(k)
 *
 * for a grid potential phi (in smooth PME, phi = theta_rec convolved with Q;
 * that FFT solve is not part of these functions). Grids are K0 x K1 x K2
 * with the last index fastest. An atom reaches the points k_a = floor(u_a) - j,
 * j = 0..n-1 (mod K_a): M_n vanishes outside (0, n). Everything in FP64.
 * ------------------------------------------------------------------------ */
double oracle_bspline(int n, double u) {
    if (n <= 2) return (u >= 0.0 && u <= 2.0) ? 1.0 - fabs(u - 1.0) : 0.0;
    return u / (n - 1) * oracle_bspline(n - 1, u) + (n - u) / (n - 1) * oracle_bspline(n - 1, u - 1.0);
}

double oracle_bspline_deriv(int n, double u) { return oracle_bspline(n - 1, u) - oracle_bspline(n - 1, u - 1.0); }

/* u in [0, K) for one coordinate */
static double pme_scaled(double x, double L, int K) {
    double s = x / L;
    s -= floor(s);
    double u = s * K;
    if (u >= K) u -= K;
    if (u < 0.0) u = 0.0;
    return u;
}

static int pme_mod(int k, int K) { return ((k % K) + K) % K; }

/*
 * Q[K0*K1*K2] = spread of the charges; Qabs (optional) the same spread of
 * |q_i| (the scale of the rounding of each grid value). Returns 0, or -1 on
 * bad arguments.
 */
int oracle_pme_spread(int n, const double *x, const double *q, const double *box, const int *K, int order, double *Q,
                      double *Qabs) {
    if (order < 2 || order > 16 || K[0] < 1 || K[1] < 1 || K[2] < 1) return -1;
    size_t ng = (size_t)K[0] * K[1] * K[2];
    memset(Q, 0, sizeof(double) * ng);
    if (Qabs) memset(Qabs, 0, sizeof(double) * ng);
    for (int i = 0; i < n; ++i) {
        double u[3], w[3][16];
        int base[3];
        for (int a = 0; a < 3; ++a) {
            u[a] = pme_scaled(x[3 * i + a], box[a], K[a]);
            base[a] = (int)floor(u[a]);
            for (int j = 0; j < order; ++j) w[a][j] = oracle_bspline(order, u[a] - (base[a] - j));
        }
        for (int j0 = 0; j0 < order; ++j0)
            for (int j1 = 0; j1 < order; ++j1)
                for (int j2 = 0; j2 < order; ++j2) {
                    size_t idx = ((size_t)pme_mod(base[0] - j0, K[0]) * K[1] + pme_mod(base[1] - j1, K[1])) * K[2] +
                                 pme_mod(base[2] - j2, K[2]);
                    double wt = w[0][j0] * w[1][j1] * w[2][j2];
                    Q[idx] += q[i] * wt;
                    if (Qabs) Qabs[idx] += fabs(q[i]) * wt;
                }
    }
    return 0;
}

/*
 * Forces F[3n] = -q_i grad psi_i for the grid potential phi, psi[n]
 * (optional) the interpolated potential of each atom, Fabs[3n] (optional)
 * the sum of |terms| of each force component. Returns 0, or -1.
 */
int oracle_pme_gather(int n, const double *x, const double *q, const double *box, const int *K, int order,
                      const double *phi, double *F, double *psi, double *Fabs) {
    if (order < 2 || order > 16 || K[0] < 1 || K[1] < 1 || K[2] < 1) return -1;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double u[3], w[3][16], dw[3][16];
        int base[3];
        for (int a = 0; a < 3; ++a) {
            u[a] = pme_scaled(x[3 * i + a], box[a], K[a]);
            base[a] = (int)floor(u[a]);
            for (int j = 0; j < order; ++j) {
                w[a][j] = oracle_bspline(order, u[a] - (base[a] - j));
                dw[a][j] = oracle_bspline_deriv(order, u[a] - (base[a] - j)) * K[a] / box[a];
            }
        }
        double f[3] = {0, 0, 0}, fa[3] = {0, 0, 0}, p = 0.0;
        for (int j0 = 0; j0 < order; ++j0)
            for (int j1 = 0; j1 < order; ++j1)
                for (int j2 = 0; j2 < order; ++j2) {
                    size_t idx = ((size_t)pme_mod(base[0] - j0, K[0]) * K[1] + pme_mod(base[1] - j1, K[1])) * K[2] +
                                 pme_mod(base[2] - j2, K[2]);
                    double ph = phi[idx];
                    double t[3] = {dw[0][j0] * w[1][j1] * w[2][j2] * ph, w[0][j0] * dw[1][j1] * w[2][j2] * ph,
                                   w[0][j0] * w[1][j1] * dw[2][j2] * ph};
                    p += w[0][j0] * w[1][j1] * w[2][j2] * ph;
                    for (int a = 0; a < 3; ++a) {
                        f[a] -= q[i] * t[a];
                        fa[a] += fabs(q[i] * t[a]);
                    }
                }
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] = f[a];
            if (Fabs) Fabs[3 * i + a] = fa[a];
        }
        if (psi) psi[i] = p;
    }
    return 0;
}

/*
 * Energies at the distances the FP32 contract fixes. E_LJ and E_C are the
 * plain FP64 definitions of pair_terms, summed over the FP32 pair set of
 * oracle_pairs_f32, each pair evaluated at its contract value
 * r^2 = fl(dz dz + fl(dy dy + fl(dx dx))), d = fl(fl(y_i - y_j) + S), y the
 * contract positions. Its difference from oracle_energy_forces (FP64
 * displacements) is the energy error that rounding the displacements to
 * FP32 causes by itself; in water the Coulomb pair energies cancel to a few
 * thousandths of their absolute sum, so at ~10^3 atoms that alone reaches
 * ~1e-6 of E_C. The cutoff is the contract's too: (float)rc, the value the
 * C ABI receives, for the pair set and for the LJ potential shift (in water
 * E_LJ cancels so far that the shift at 0.9 and at (float)0.9 give E_LJ
 * values ~2e-6 apart). E[0] = E_LJ, E[1] = E_C, E[2] and E[3] the sums of
 * |e_LJ| and |e_C| over the pairs. Returns 0, or the error code of
 * oracle_pairs_f32 (-2: out of memory).
 */
int oracle_energy_f32(int n, const float *x0, const float *x, const double *q, const int *type, int ntype,
                      const double *lj, const float *box, double rc, double beta, const int *excl_off,
                      const int *excl_idx, double *E, long long *npairs) {
    const float rcf = (float)rc;
    long long cnt = 0;
    int st = oracle_pairs_f32(n, x0, x, box, rcf, excl_off, excl_idx, NULL, NULL, 0, &cnt);
    if (st < 0) return st;
    int *pi = (int *)malloc(sizeof(int) * (size_t)(cnt + 1));
    int *pj = (int *)malloc(sizeof(int) * (size_t)(cnt + 1));
    float *y = (float *)malloc(sizeof(float) * 3 * (size_t)n + 1);
    if (!pi || !pj || !y) {
        free(pi);
        free(pj);
        free(y);
        return -2;
    }
    st = oracle_pairs_f32(n, x0, x, box, rcf, excl_off, excl_idx, pi, pj, cnt, &cnt);
    oracle_image_f32(n, x0, x, box, y);
    const float rc2 = rcf * rcf;
    double sum_lj = 0.0, sum_c = 0.0, abs_lj = 0.0, abs_c = 0.0;
    for (long long p = 0; st >= 0 && p < cnt; ++p) {
        const int i = pi[p], j = pj[p];
        float u[3];
        for (int k = 0; k < 3; ++k) u[k] = y[3 * i + k] - y[3 * j + k];
        for (int sx = -1; sx <= 1; ++sx)
            for (int sy = -1; sy <= 1; ++sy)
                for (int sz = -1; sz <= 1; ++sz) {
                    const float dx = u[0] + (float)sx * box[0];
                    const float dy = u[1] + (float)sy * box[1];
                    const float dz = u[2] + (float)sz * box[2];
                    const float r2 = r2_32(dx, dy, dz);
                    if (!(r2 < rc2)) continue;  /* the one image within rc (the pair set checks it) */
                    const double *c = lj + 2 * ((size_t)type[i] * ntype + type[j]);
                    double elj, ec, s;
                    pair_terms((double)r2, q[i], q[j], c[0], c[1], (double)rcf, beta, &elj, &ec, &s);
                    sum_lj += elj;
                    sum_c += ec;
                    abs_lj += fabs(elj);
                    abs_c += fabs(ec);
                }
    }
    E[0] = sum_lj;
    E[1] = sum_c;
    E[2] = abs_lj;
    E[3] = abs_c;
    *npairs = cnt;
    free(pi);
    free(pj);
    free(y);
    return st < 0 ? st : 0;
}
