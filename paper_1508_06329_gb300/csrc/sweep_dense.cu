// sweep_dense.cu — one sweep of multi-sweep LexBFS on a dense graph: LexBFS
// whose ties go to a caller-given rank (or to the vertex latest in a previous
// sweep: LexBFS+), optionally from a given start vertex.
//
// Method: LexBFS of Section 4.2 numbers, among the vertices with the
// lexicographically largest label, the first one of the top class; with the
// single initial class ordered by rank, that is the one of smallest rank.
// Labels do not depend on vertex names, so the sweep equals the lowest-id
// LexBFS of the graph relabelled v -> newid(v) (newid = position in the order
// start first, then by rank), mapped back.  The GPU form therefore is
//   1. ids:     newid[v] and inv[newid] = v from the tie-break array;
//   2. permute: the relabelled bit matrix, one CTA per new row (the old row's
//               set bits scattered to their new columns in shared memory);
//   3. the LexBFS kernel on the relabelled matrix;
//   4. unpermute: order[i] = inv[order'[i]], pos[v] = pos'[newid[v]].
// Every index read from caller data is range-checked before use, so an
// invalid tie-break array (not a permutation) yields an unspecified order and
// a flag (checked on the host when validation is on), never a stray access.
#include <algorithm>

#include "kernels.h"

namespace cg {

namespace {

// rank of every vertex into rankv[] (kind RANK: tb[v]; kind LAST_IN: tb is a
// previous order, the vertex at position i gets rank n - 1 - i; kind ID: v).
// seen[] (zeroed) detects repeated ranks / vertices.
__global__ void sweep_rank_kernel(int n, int kind, const int32_t *__restrict__ tb, int32_t *__restrict__ rankv,
                                  int *__restrict__ seen, int *__restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int v = i, r = i;
        if (kind == CG_TIE_RANK) {
            r = tb[i];
        } else if (kind == CG_TIE_LAST_IN) {
            v = tb[i];
            r = n - 1 - i;
        }
        if (v < 0 || v >= n || r < 0 || r >= n || atomicExch(&seen[r], 1) != 0) {
            atomicOr(flag, 1);
            continue;
        }
        rankv[v] = r;
    }
}

// start first, then by rank: newid = rank + (rank < rank(start)); inv = newid^-1
// (inv zeroed beforehand, so that it stays in range for invalid input)
__global__ void sweep_ids_kernel(int n, int start, const int32_t *__restrict__ rankv, int32_t *__restrict__ newid,
                                 int32_t *__restrict__ inv) {
    int rs = start >= 0 ? rankv[start] : 0;
    if (rs < 0 || rs >= n) rs = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int r = rankv[v];
        if (r < 0 || r >= n) r = 0;   // invalid input (flagged): keep every index in range
        if (start >= 0) r = v == start ? 0 : r + (r < rs ? 1 : 0);
        newid[v] = r;
        inv[r] = v;
    }
}

// New row r is old row inv[r] with column j moved to newid[j].
__global__ void sweep_permute_kernel(int n, const uint32_t *__restrict__ rows, int words_in,
                                     const int32_t *__restrict__ newid, const int32_t *__restrict__ inv,
                                     uint32_t *__restrict__ out) {
    extern __shared__ uint32_t srow[];
    const int wn = (n + 31) >> 5;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        for (int w = threadIdx.x; w < wn; w += blockDim.x) srow[w] = 0u;
        __syncthreads();
        const int v = __ldg(inv + r);
        const uint32_t *src = rows + (size_t)v * words_in;
        for (int w = threadIdx.x; w < wn; w += blockDim.x) {
            uint32_t bits = __ldg(src + w);
            if (w == wn - 1 && (n & 31)) bits &= (1u << (n & 31)) - 1u;
            while (bits) {
                const int j = (w << 5) + __ffs(bits) - 1;
                bits &= bits - 1;
                const int nj = __ldg(newid + j);
                if (nj != r) atomicOr(&srow[nj >> 5], 1u << (nj & 31));   // no loop even for invalid input
            }
        }
        __syncthreads();
        uint32_t *dst = out + (size_t)r * wn;
        for (int w = threadIdx.x; w < wn; w += blockDim.x) dst[w] = srow[w];
        __syncthreads();
    }
}

__global__ void sweep_unpermute_kernel(int n, const int32_t *__restrict__ newid, const int32_t *__restrict__ inv,
                                       const int32_t *__restrict__ order_p, const int32_t *__restrict__ pos_p,
                                       int32_t *__restrict__ order, int32_t *__restrict__ pos) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = order_p[i];
        order[i] = inv[x];
        if (pos) pos[i] = pos_p[newid[i]];
    }
}

}  // namespace

int sweep_ids_launch(int n, int kind, const int32_t *tiebreak, int start, const SweepBuffers &sb, int num_sms,
                     cudaStream_t stream) {
    if (n <= 0) return CG_OK;
    const int blocks = (int)std::min<int64_t>(ceil_div((int64_t)n, 256), (int64_t)num_sms * 4);
    CG_CUDA_TRY(cudaMemsetAsync(sb.seen, 0, (size_t)n * 4, stream));
    CG_CUDA_TRY(cudaMemsetAsync(sb.rankv, 0xFF, (size_t)n * 4, stream));
    CG_CUDA_TRY(cudaMemsetAsync(sb.inv, 0, (size_t)n * 4, stream));
    CG_CUDA_TRY(cudaMemsetAsync(sb.flag, 0, sizeof(int), stream));
    sweep_rank_kernel<<<blocks, 256, 0, stream>>>(n, kind, tiebreak, sb.rankv, sb.seen, sb.flag);
    CG_LAUNCH_CHECK("sweep_rank_kernel");
    sweep_ids_kernel<<<blocks, 256, 0, stream>>>(n, start, sb.rankv, sb.newid, sb.inv);
    CG_LAUNCH_CHECK("sweep_ids_kernel");
    return CG_OK;
}

int sweep_unpermute_launch(int n, const SweepBuffers &sb, int32_t *order, int32_t *pos, int num_sms,
                           cudaStream_t stream) {
    if (n <= 0) return CG_OK;
    const int blocks = (int)std::min<int64_t>(ceil_div((int64_t)n, 256), (int64_t)num_sms * 4);
    sweep_unpermute_kernel<<<blocks, 256, 0, stream>>>(n, sb.newid, sb.inv, sb.order_p, sb.pos_p, order, pos);
    CG_LAUNCH_CHECK("sweep_unpermute_kernel");
    return CG_OK;
}

int sweep_order_launch(const DenseDesc &d, const LexPlan &plan, void *gstate, int *counter, const SweepBuffers &sb,
                       int32_t *order, int32_t *pos, int num_sms, cudaStream_t stream) {
    const int n = d.n;
    if (n <= 0) return CG_OK;
    const int wn = (n + 31) / 32;
    const int blocks = (int)std::min<int64_t>(ceil_div((int64_t)n, 256), (int64_t)num_sms * 4);
    const int pthreads = wn >= 256 ? 512 : 128;
    sweep_permute_kernel<<<std::min(n, num_sms * 8), pthreads, (size_t)wn * 4, stream>>>(n, d.rows, d.words,
                                                                                         sb.newid, sb.inv, sb.prow);
    CG_LAUNCH_CHECK("sweep_permute_kernel");
    DenseDesc dp = d;
    dp.rows = sb.prow;
    dp.words = wn;
    int rc = lexbfs_dense_launch(plan, nullptr, dp, 1, 1, sb.order_p, sb.pos_p, nullptr, gstate, counter, stream);
    if (rc) return rc;
    sweep_unpermute_kernel<<<blocks, 256, 0, stream>>>(n, sb.newid, sb.inv, sb.order_p, sb.pos_p, order, pos);
    CG_LAUNCH_CHECK("sweep_unpermute_kernel");
    return CG_OK;
}

}  // namespace cg
