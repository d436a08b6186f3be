// nb_forces_noalloc: pair search plus forces for small systems, with every
// scratch buffer carved out of one statically allocated device array, so
// that the call allocates no device memory. Declared in include/nb.h.
//
// The array is a file-scope __device__ variable: each GPU that loads this
// library holds it until the process exits. Host code cannot use its name
// as a device address, so the first call on each device looks the address
// up with cudaGetSymbolAddress (with that device current) and keeps it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "nb_internal.cuh"

namespace {

constexpr int kMaxAtoms = NB_NOALLOC_MAX_ATOMS;
constexpr int kMaxClus = (kMaxAtoms + NB_CLUSTER - 1) / NB_CLUSTER;  // clusters of real atoms
constexpr int kMaxCols = kMaxClus;                                    // grid columns
constexpr int kMaxNc = kMaxClus + kMaxCols;                           // clusters incl. padding
constexpr int kMaxSlots = kMaxNc * NB_CLUSTER;
// List entries: one per cluster pair of a full half list, twice over. In a
// cubic 4,096-atom water box with rc one float below L/2 (the largest cutoff
// the call takes) the half list holds about 1.1 entries per cluster pair (a
// pair can be listed under two shifts), so this leaves room to spare.
constexpr size_t kCapEntries = (size_t)kMaxClus * kMaxClus;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte layout of the scratch array (each piece 256-byte aligned).
constexpr size_t kOffState = 0;
constexpr size_t kOffColCount = kOffState + align256(sizeof(nb_dev_state));
constexpr size_t kOffColAtom = kOffColCount + align256(sizeof(int) * kMaxCols);
constexpr size_t kOffColClus = kOffColAtom + align256(sizeof(int) * (kMaxCols + 1));
constexpr size_t kOffAtomCol = kOffColClus + align256(sizeof(int) * (kMaxCols + 1));
constexpr size_t kOffAtomSlot = kOffAtomCol + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffXw = kOffAtomSlot + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffKeys = kOffXw + align256(sizeof(float4) * kMaxAtoms);
constexpr size_t kOffPerm = kOffKeys + align256(sizeof(unsigned long long) * kMaxAtoms);
constexpr size_t kOffPos = kOffPerm + align256(sizeof(int) * kMaxSlots);
constexpr size_t kOffXref = kOffPos + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffXprune = kOffXref + align256(sizeof(float4) * kMaxSlots);
constexpr size_t kOffXq = kOffXprune + align256(sizeof(float4) * kMaxSlots);
constexpr size_t kOffTsort = kOffXq + align256(sizeof(float4) * kMaxSlots);
constexpr size_t kOffFsort = kOffTsort + align256(sizeof(int) * kMaxSlots);
constexpr size_t kOffBbox = kOffFsort + align256(sizeof(float4) * kMaxSlots);
constexpr size_t kOffList = kOffBbox + align256(sizeof(float4) * 2 * kMaxNc);
constexpr size_t kOffCiStart = kOffList + align256(sizeof(int4) * kCapEntries);
constexpr size_t kOffCiLenO = kOffCiStart + align256(sizeof(int) * kMaxNc);
constexpr size_t kOffCiLenI = kOffCiLenO + align256(sizeof(int) * kMaxNc);
constexpr size_t kOffSys = kOffCiLenI + align256(sizeof(int) * kMaxNc);
constexpr size_t kOffShift = kOffSys + align256(sizeof(nb_sys));
constexpr size_t kOffAtomSys = kOffShift + align256(sizeof(float4) * 27);
constexpr size_t kOffColSys = kOffAtomSys + align256(sizeof(int) * kMaxAtoms);
constexpr size_t kOffClusSys = kOffColSys + align256(sizeof(int) * kMaxCols);
constexpr size_t kOffZtab = kOffClusSys + align256(sizeof(int) * kMaxNc);
constexpr size_t kScratchBytes = kOffZtab + align256(sizeof(int) * kMaxCols * (NB_ZBINS + 1));

static_assert(kScratchBytes == NB_NOALLOC_SCRATCH_BYTES, "update NB_NOALLOC_SCRATCH_BYTES in nb.h");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

int fail(int code, const char *what) { return nb_record_error(code, what); }

}  // namespace

extern "C" int nb_forces_noalloc(int n_atoms, const float *coords, const float *box, const float *q,
                                 const int *type, int ntype, const float *ljparams, float rc, float beta,
                                 const int *excl_off, const int *excl_idx, float *forces, double *energies,
                                 unsigned *error_word, void *stream) {
    if (n_atoms < 1) return fail(NB_ERR_ARG, "nb_forces_noalloc: n_atoms < 1");
    if (n_atoms > kMaxAtoms)
        return fail(NB_ERR_CAPACITY, "nb_forces_noalloc: n_atoms exceeds NB_NOALLOC_MAX_ATOMS (4096)");
    if (!coords || !box || !q || !type || !ljparams || !forces)
        return fail(NB_ERR_ARG, "nb_forces_noalloc: NULL argument");
    if ((excl_off == nullptr) != (excl_idx == nullptr))
        return fail(NB_ERR_ARG, "nb_forces_noalloc: give both exclusion arrays or neither");
    if (ntype < 1 || ntype > NB_MAX_TYPES) return fail(NB_ERR_ARG, "nb_forces_noalloc: ntype not in [1, 32]");
    if (!(rc > 0.0f) || !(beta >= 0.0f) || !((double)beta * rc <= 3.2))
        return fail(NB_ERR_ARG, "nb_forces_noalloc: need rc > 0 and 0 <= beta*rc <= 3.2");
    for (int k = 0; k < 3; ++k)
        if (!(box[k] > 2.0f * rc) || !(box[k] < 3.0e38f))
            return fail(NB_ERR_ARG, "nb_forces_noalloc: each box edge must exceed 2*rc");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(NB_ERR_CUDA, "nb_forces_noalloc: no usable current device");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p)
                return fail(NB_ERR_CUDA, "nb_forces_noalloc: cudaGetSymbolAddress of the scratch array failed");
            g_scratch_addr[dev] = (unsigned char *)p;
        }
        base = g_scratch_addr[dev];
    }

    // A pair list whose buffers all point into the scratch array, sized for
    // the maximum system; nothing here allocates.
    nb_pairlist pl;
    std::memset(&pl, 0, sizeof(pl));
    pl.device = dev;
    if (cudaDeviceGetAttribute(&pl.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(NB_ERR_CUDA, "nb_forces_noalloc: cudaDeviceGetAttribute failed");
    const int nclus = (n_atoms + NB_CLUSTER - 1) / NB_CLUSTER;
    pl.n_atoms = n_atoms;
    pl.ncol_max = nclus;
    pl.nc_max = 2 * nclus;
    pl.cap = kCapEntries;
    pl.st = (nb_dev_state *)(base + kOffState);
    pl.col_count = (int *)(base + kOffColCount);
    pl.col_atom_start = (int *)(base + kOffColAtom);
    pl.col_clus_start = (int *)(base + kOffColClus);
    pl.atom_col = (int *)(base + kOffAtomCol);
    pl.atom_slot = (int *)(base + kOffAtomSlot);
    pl.xw = (float4 *)(base + kOffXw);
    pl.keys = (unsigned long long *)(base + kOffKeys);
    pl.perm = (int *)(base + kOffPerm);
    pl.pos = (int *)(base + kOffPos);
    pl.xref = (float4 *)(base + kOffXref);
    pl.xprune = (float4 *)(base + kOffXprune);
    pl.xq = (float4 *)(base + kOffXq);
    pl.tsort = (int *)(base + kOffTsort);
    pl.fsort = (float4 *)(base + kOffFsort);
    pl.bbox = (float4 *)(base + kOffBbox);
    pl.outer = (int4 *)(base + kOffList);
    pl.inner = pl.outer;  // no prune in this call
    pl.ci_start = (int *)(base + kOffCiStart);
    pl.ci_len_outer = (int *)(base + kOffCiLenO);
    pl.ci_len_inner = (int *)(base + kOffCiLenI);
    pl.nsys = 1;
    pl.sys = (nb_sys *)(base + kOffSys);
    pl.sys_shift = (float4 *)(base + kOffShift);
    pl.atom_sys = (int *)(base + kOffAtomSys);
    pl.col_sys = (int *)(base + kOffColSys);
    pl.clus_sys = (int *)(base + kOffClusSys);
    pl.ztab = (int *)(base + kOffZtab);
    for (int k = 0; k < 3; ++k) pl.box[k] = box[k];

    // same grid rule as nb_search
    const double Lx = box[0], Ly = box[1], Lz = box[2];
    const double side = std::cbrt(NB_CLUSTER * Lx * Ly * Lz / (double)n_atoms);
    int ncx = std::max(1, (int)std::floor(Lx / side)), ncy = std::max(1, (int)std::floor(Ly / side));
    while ((long long)ncx * ncy > pl.ncol_max) {
        if (ncx >= ncy) --ncx; else --ncy;
    }
    pl.ncx = ncx;
    pl.ncy = ncy;
    pl.ncol = ncx * ncy;

    cudaStream_t s = (cudaStream_t)stream;
    // The scratch keeps the previous call's contents: reset the state block
    // (error word, counters, cluster count) and the atom -> slot map, which
    // the permute-back reads for every atom.
    if (cudaMemsetAsync(pl.st, 0, sizeof(nb_dev_state), s) != cudaSuccess ||
        cudaMemsetAsync(pl.pos, 0, sizeof(int) * (size_t)n_atoms, s) != cudaSuccess ||
        cudaMemsetAsync(pl.atom_sys, 0, sizeof(int) * (size_t)n_atoms, s) != cudaSuccess ||
        cudaMemsetAsync(pl.col_sys, 0, sizeof(int) * (size_t)pl.ncol, s) != cudaSuccess)
        return fail(NB_ERR_CUDA, "nb_forces_noalloc: cudaMemsetAsync failed");
    nb_sys one;
    std::memset(&one, 0, sizeof(one));
    one.box = make_float4(box[0], box[1], box[2], 0.0f);
    one.inv_sx = (float)(ncx / Lx);
    one.inv_sy = (float)(ncy / Ly);
    one.ncx = ncx;
    one.ncy = ncy;
    one.n_atoms = n_atoms;
    const float lmax = std::max(box[0], std::max(box[1], box[2]));
    const double ulp = (double)std::nextafter(lmax, 2.0f * lmax) - lmax;
    const double rle = rc + std::max(1e-5, 8.0 * ulp) + 1e-6 * rc;
    const float rl2 = std::nextafter((float)(rle * rle), 1e30f);
    cudaError_t e = nb_launch_grid_sort(&pl, coords, &one, s);
    if (e == cudaSuccess) e = nb_launch_search(&pl, excl_off, excl_idx, rl2, (float)(rle + 1e-3), s);
    pl.searched = 1;
    pl.has_inner = 0;
    pl.rlist = rc;
    if (e == cudaSuccess) e = nb_launch_gather(&pl, coords, q, type, ntype, 0, energies, NB_PART_ALL, s);
    if (e == cudaSuccess) e = nb_launch_force(&pl, ntype, ljparams, rc, beta, energies, 0.0f, 0.0f, NB_PART_ALL, s);
    if (e == cudaSuccess) e = nb_launch_scatter(&pl, forces, s);
    if (e != cudaSuccess) return fail(NB_ERR_CUDA, cudaGetErrorString(e));
    if (error_word) {
        if (cudaMemcpyAsync(error_word, &pl.st->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(NB_ERR_CUDA, "nb_forces_noalloc: reading the error word failed");
    }
    return NB_OK;
}
