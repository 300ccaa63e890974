// gs_radix.cuh -- stable LSD radix passes over (key, value) pairs of int32,
// 8 bits per pass, for the atom cell list: keys are cell indices, values
// atom indices, and the pairs enter in atom order (values omitted: the
// identity), so after the passes the atoms are grouped by cell in ascending
// atom order within each cell.  Every pass reads and writes each pair once,
// so the time is bounded by the number of atoms for any distribution of
// atoms over cells (a crowded cell costs no more than a spread-out one).
//
// A pass: rs_hist counts the digits of each block's RS_TILE pairs into
// hist[digit * nblk + block]; an exclusive scan of hist (digit-major) gives
// each (digit, block) its first output slot; rs_scatter writes each pair to
// that slot plus its rank among the block's pairs with the same digit,
// taken in input order (warp match + per-warp counts), which keeps the
// sort stable.
#pragma once
#include "gs_internal.cuh"

#define RS_THREADS 256
#define RS_ROUNDS 8
#define RS_TILE (RS_THREADS * RS_ROUNDS)

// passes needed for keys in [0, nkeys)
__host__ __forceinline__ int rs_passes(int64_t nkeys)
{
    int bits = 0;
    while (bits < 32 && (((int64_t)1 << bits) < nkeys)) bits++;
    return (bits + 7) / 8;
}

template <typename OFF>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const int32_t *__restrict__ keys, int64_t n, int shift,
                                                         OFF *__restrict__ hist, int64_t nblk)
{
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ROUNDS; j++) {
        const int64_t i = base + (int64_t)j * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = (OFF)h[threadIdx.x];
}

// vals_in null: the value of pair i is i; keys_out null: keys not kept
template <typename OFF>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const int32_t *__restrict__ keys_in,
                                                            const int32_t *__restrict__ vals_in, int64_t n, int shift,
                                                            const OFF *__restrict__ offs, int64_t nblk,
                                                            int32_t *__restrict__ keys_out,
                                                            int32_t *__restrict__ vals_out)
{
    constexpr int NW = RS_THREADS / 32;
    __shared__ int64_t run[256];
    __shared__ int32_t wcnt[NW][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = (int64_t)offs[(int64_t)threadIdx.x * nblk + blockIdx.x];
    for (int k = threadIdx.x; k < NW * 256; k += RS_THREADS) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int j = 0; j < RS_ROUNDS; j++) {
        const int64_t i = base + (int64_t)j * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        const int32_t key = valid ? keys_in[i] : 0;
        const unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        const bool leader = rank == 0;
        if (valid && leader) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = run[d] + rank;
            for (int q = 0; q < w; q++) pos += wcnt[q][d];
            vals_out[pos] = vals_in ? vals_in[i] : (int32_t)i;
            if (keys_out) keys_out[pos] = key;
        }
        __syncthreads();
        {
            const int dd = threadIdx.x;  // one thread per digit
            int32_t tot = 0;
            for (int q = 0; q < NW; q++) { tot += wcnt[q][dd]; wcnt[q][dd] = 0; }
            run[dd] += tot;
        }
        __syncthreads();
    }
}

static __global__ void k_rs_iota(int32_t *__restrict__ v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}
