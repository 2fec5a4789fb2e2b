// Kendall discordant-pair counts for the MMD test of Sec. 5 (Mallows kernel).
//
// For each pair p of permutations (s, t) = (perms[2p], perms[2p + 1]) of
// [0, n), n_dis = #{i < j : (s_i < s_j) != (t_i < t_j)}.  One CTA owns one
// pair at a time: both permutations are staged in shared memory, every
// thread takes rows i (strided) and counts the discordant j > i, and a block
// reduction gives the count.  O(n^2) comparisons per pair, all in shared
// memory; the pairs are independent.
#include <cstdint>

#include "bshuffle_internal.h"

namespace bsh {
namespace {

constexpr int kKBlock = 256;
constexpr uint32_t kMaxN = 4096;

__global__ void __launch_bounds__(kKBlock) kendall_pairs_kernel(const uint32_t *__restrict__ perms, uint32_t n,
                                                                uint64_t pairs, uint64_t *__restrict__ out)
{
    __shared__ uint32_t s_a[kMaxN];
    __shared__ uint32_t s_b[kMaxN];
    __shared__ unsigned long long s_sum[kKBlock / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    for (uint64_t p = blockIdx.x; p < pairs; p += gridDim.x) {
        const uint32_t *a = perms + 2 * p * n;
        const uint32_t *b = a + n;
        for (uint32_t i = tid; i < n; i += kKBlock) {
            s_a[i] = a[i];
            s_b[i] = b[i];
        }
        __syncthreads();
        unsigned long long count = 0;
        // rows i and n-1-i together keep the work per thread balanced
        for (uint32_t i = tid; i < (n + 1) / 2; i += kKBlock) {
            for (uint32_t r = 0; r < 2; ++r) {
                const uint32_t row = r == 0 ? i : n - 1 - i;
                if (r == 1 && row == i) break;
                const uint32_t ai = s_a[row], bi = s_b[row];
                uint32_t c = 0;
                for (uint32_t j = row + 1; j < n; ++j) c += ((ai < s_a[j]) != (bi < s_b[j])) ? 1u : 0u;
                count += c;
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) count += __shfl_down_sync(0xffffffffu, count, d);
        if (lane == 0) s_sum[warp] = count;
        __syncthreads();
        if (tid == 0) {
            unsigned long long total = 0;
            for (int w = 0; w < kKBlock / 32; ++w) total += s_sum[w];
            out[p] = total;
        }
        __syncthreads();
    }
}

// sigma[r][idx[r][j]] = j for every row r: a shuffle's slot order (element
// idx[j] in slot j) turned into the rank of each element, the permutation
// convention of Sec. 2.
__global__ void __launch_bounds__(kKBlock) invert_rows_kernel(const uint32_t *__restrict__ idx, uint32_t n,
                                                              uint64_t rows, uint32_t *__restrict__ sigma)
{
    const uint64_t total = rows * n;
    for (uint64_t e = static_cast<uint64_t>(blockIdx.x) * kKBlock + threadIdx.x; e < total;
         e += static_cast<uint64_t>(gridDim.x) * kKBlock) {
        const uint64_t r = e / n;
        const uint32_t j = static_cast<uint32_t>(e - r * n);
        const uint32_t v = idx[e];
        if (v < n) sigma[r * n + v] = j;
    }
}

}  // namespace

uint32_t kendall_max_n() { return kMaxN; }

cudaError_t launch_invert_rows(const uint32_t *idx, uint32_t n, uint64_t rows, uint32_t *sigma, cudaStream_t stream)
{
    int device = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (rows * n + kKBlock - 1) / kKBlock;
    const uint64_t grid = blocks < static_cast<uint64_t>(sms) * 16 ? blocks : static_cast<uint64_t>(sms) * 16;
    invert_rows_kernel<<<static_cast<unsigned>(grid), kKBlock, 0, stream>>>(idx, n, rows, sigma);
    return cudaGetLastError();
}

cudaError_t launch_kendall_pairs(const uint32_t *perms, uint32_t n, uint64_t pairs, uint64_t *out,
                                 cudaStream_t stream)
{
    int device = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const uint64_t grid = pairs < static_cast<uint64_t>(sms) * 8 ? pairs : static_cast<uint64_t>(sms) * 8;
    kendall_pairs_kernel<<<static_cast<unsigned>(grid), kKBlock, 0, stream>>>(perms, n, pairs, out);
    return cudaGetLastError();
}

}  // namespace bsh
