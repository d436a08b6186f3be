// Post-prune list sorting (§III-A: the HIP fork's "post-pruning list
// sorting strategy" that cuts the tail of the NBNXM and prune kernels, with
// the prune computing a "list size histogram").
//
// The force kernel hands out i-clusters from a work counter; taking them in
// order of decreasing list length lets the longest lists start first, so the
// persistent grid ends with short items and a short tail.
//
// k_len_hist     histogram of the per-i-cluster list lengths (after a search;
//                after a prune the prune kernel builds it, as in the paper)
// k_len_offsets  exclusive scan of the histogram from the longest length down
// k_len_scatter  ci -> order[offset(len) + rank within its length]
#include "nb_internal.cuh"

namespace {

// Both kernels aggregate in shared memory first: the lengths of many
// clusters fall in a few bins, and global atomics on one address serialise.
constexpr int kSortThreads = 256;

__global__ void __launch_bounds__(kSortThreads) k_len_hist(const int *__restrict__ ci_len, const nb_dev_state *st,
                                                           int *__restrict__ hist) {
    __shared__ int s_cnt[NB_LEN_BINS];
    const int nc = st->nc;
    for (int b = threadIdx.x; b < NB_LEN_BINS; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    for (int ci = blockIdx.x * blockDim.x + threadIdx.x; ci < nc; ci += gridDim.x * blockDim.x)
        atomicAdd(&s_cnt[min(ci_len[ci], NB_LEN_BINS - 1)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < NB_LEN_BINS; b += blockDim.x)
        if (s_cnt[b] > 0) atomicAdd(&hist[b], s_cnt[b]);
}

// One CTA of NB_LEN_BINS threads: offsets[len] = number of clusters with a
// longer list.
__global__ void __launch_bounds__(NB_LEN_BINS) k_len_offsets(const int *__restrict__ hist, int *__restrict__ offsets,
                                                           int *__restrict__ cursor) {
    __shared__ int s[NB_LEN_BINS];
    nb_pdl_wait();
    nb_pdl_release();
    const int t = threadIdx.x;
    s[t] = hist[NB_LEN_BINS - 1 - t];  // reversed: longest first
    __syncthreads();
    for (int o = 1; o < NB_LEN_BINS; o <<= 1) {
        const int v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    const int len = NB_LEN_BINS - 1 - t;
    offsets[len] = s[t] - hist[len];  // exclusive
    cursor[len] = 0;
}

// Each pass of a CTA places kSortThreads clusters: ranks within the CTA by
// shared atomics, then one global atomic per occupied bin reserves the
// CTA's places in that bin.
__global__ void __launch_bounds__(kSortThreads) k_len_scatter(const int *__restrict__ ci_len, const nb_dev_state *st,
                                                              const int *__restrict__ offsets,
                                                              int *__restrict__ cursor, int *__restrict__ order) {
    __shared__ int s_cnt[NB_LEN_BINS];
    __shared__ int s_base[NB_LEN_BINS];
    nb_pdl_wait();
    nb_pdl_release();
    const int nc = st->nc;
    for (int c0 = blockIdx.x * blockDim.x; c0 < nc; c0 += gridDim.x * blockDim.x) {
        for (int b = threadIdx.x; b < NB_LEN_BINS; b += blockDim.x) s_cnt[b] = 0;
        __syncthreads();
        const int ci = c0 + (int)threadIdx.x;
        const int len = ci < nc ? min(ci_len[ci], NB_LEN_BINS - 1) : 0;
        const int rank = ci < nc ? atomicAdd(&s_cnt[len], 1) : 0;
        __syncthreads();
        for (int b = threadIdx.x; b < NB_LEN_BINS; b += blockDim.x)
            if (s_cnt[b] > 0) s_base[b] = atomicAdd(&cursor[b], s_cnt[b]);
        __syncthreads();
        if (ci < nc) order[offsets[len] + s_base[len] + rank] = ci;
        __syncthreads();
    }
}

}  // namespace

cudaError_t nb_clear_len_hist(nb_pairlist *pl, cudaStream_t s) {
    return cudaMemsetAsync(pl->len_hist, 0, sizeof(int) * NB_LEN_BINS, s);
}

cudaError_t nb_launch_sort_by_length(nb_pairlist *pl, const int *ci_len, bool hist_ready, cudaStream_t s) {
    const int blocks = max(1, min((pl->nc_max + kSortThreads - 1) / kSortThreads, pl->num_sms * 4));
    if (!hist_ready) {
        cudaError_t e = nb_clear_len_hist(pl, s);
        if (e != cudaSuccess) return e;
        k_len_hist<<<blocks, kSortThreads, 0, s>>>(ci_len, pl->st, pl->len_hist);
    }
    cudaError_t e = nb_launch_pdl(k_len_offsets, 1, NB_LEN_BINS, 0, s, (const int *)pl->len_hist, pl->len_offsets,
                                  pl->len_cursor);
    if (e != cudaSuccess) return e;
    return nb_launch_pdl(k_len_scatter, blocks, kSortThreads, 0, s, ci_len, (const nb_dev_state *)pl->st,
                         (const int *)pl->len_offsets, pl->len_cursor, pl->ci_order);
}
