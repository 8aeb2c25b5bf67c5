// sweep_csr.cu — one sweep of multi-sweep LexBFS on a CSR graph (tie-break
// rank or LexBFS+ of a previous sweep, optional start vertex).
//
// As for dense graphs (sweep_dense.cu), the sweep is the lowest-id LexBFS of
// the graph relabelled v -> newid(v), mapped back.  Relabelling a CSR graph
// means: new row r = old row inv[r] with every column c replaced by newid[c]
// and the row sorted again (the CSR LexBFS keeps its class member lists in
// row order).  GPU form:
//   1. new ids (sweep_ids_launch, shared with the dense sweep);
//   2. degrees of the new rows and an exclusive scan -> the new row_ptr;
//   3. the rows sorted by size class: up to 32 entries one warp (a bitonic
//      network over the lanes), up to kMidMax one CTA (bitonic in shared
//      memory), longer rows one CTA each on a power-of-two padded copy in the
//      workspace (bitonic passes separated by __syncthreads);
//   4. the CSR LexBFS kernel on the relabelled copy;
//   5. order[i] = inv[order'[i]], pos[v] = pos'[newid[v]].
#include <algorithm>
#include <climits>

#include "kernels.h"

namespace cg {

namespace {

constexpr int kMidMax = 4096;      // longest row sorted in shared memory
constexpr int kScanTile = 1024;    // elements per CTA of the scan (256 threads x 4)

// ---- exclusive scan of int64 values: out[0..count] (out[count] = total)

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t *warp_sums, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    const int64_t before = warp > 0 ? warp_sums[warp - 1] : 0;
    if (total) *total = warp_sums[nw - 1];
    __syncthreads();
    return before + incl - x;
}

__global__ void scan_tiles_kernel(const int64_t *__restrict__ in, int64_t count, int64_t *__restrict__ out,
                                  int64_t *__restrict__ tile_sums) {
    __shared__ int64_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 4;
    int64_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < count ? in[base + k] : 0;
        s += v[k];
    }
    int64_t tot;
    int64_t run = block_exclusive_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < count) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// one CTA: exclusive scan of the tile sums in chunks, carrying the running total
__global__ void scan_sums_kernel(int64_t *__restrict__ tile_sums, int64_t tiles, int64_t *__restrict__ total_out) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < tiles; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const int64_t x = i < tiles ? tile_sums[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(x, ws, &tot);
        if (i < tiles) tile_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void scan_add_kernel(int64_t *__restrict__ out, int64_t count, const int64_t *__restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int64_t add = tile_sums[blockIdx.x];
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
        if (base + k < count) out[base + k] += add;
}

int scan_launch(const int64_t *in, int64_t count, int64_t *out, int64_t *tile_sums, cudaStream_t stream) {
    const int64_t tiles = std::max<int64_t>(1, ceil_div(count, kScanTile));
    if (tiles > INT_MAX) return set_error(CG_EINVAL, "scan too long");
    scan_tiles_kernel<<<(int)tiles, 256, 0, stream>>>(in, count, out, tile_sums);
    CG_LAUNCH_CHECK("scan_tiles_kernel");
    scan_sums_kernel<<<1, 1024, 0, stream>>>(tile_sums, tiles, out + count);
    CG_LAUNCH_CHECK("scan_sums_kernel");
    scan_add_kernel<<<(int)tiles, 256, 0, stream>>>(out, count, tile_sums);
    CG_LAUNCH_CHECK("scan_add_kernel");
    return CG_OK;
}

// ---- the relabelled rows

__host__ __device__ inline int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// degree of every new row, and the padded length of the rows sorted in the workspace
__global__ void sweep_csr_degrees_kernel(int n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ inv,
                                         int64_t *__restrict__ deg, int64_t *__restrict__ padded) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int u = inv[r];
        const int64_t d = row_ptr[u + 1] - row_ptr[u];
        deg[r] = d;
        padded[r] = d > kMidMax ? next_pow2(d) : 0;
    }
}

// rows of at most 32 entries: one warp each, a bitonic network over the lanes
__global__ void sweep_csr_small_kernel(int n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                       const int32_t *__restrict__ newid, const int32_t *__restrict__ inv,
                                       const int64_t *__restrict__ rp_new, int32_t *__restrict__ col_new) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
        const int64_t d = rp_new[r + 1] - rp_new[r];
        if (d > 32) continue;
        const int u = inv[r];
        int x = lane < d ? newid[col[row_ptr[u] + lane]] : INT_MAX;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
                const bool up = (lane & k) == 0, low = (lane & j) == 0;
                x = (up == low) ? min(x, y) : max(x, y);
            }
        }
        if (lane < d) col_new[rp_new[r] + lane] = x;
    }
}

// bitonic sort of a[0..p) (p a power of two) by one CTA
__device__ void cta_bitonic(int32_t *a, int64_t p) {
    for (int64_t k = 2; k <= p; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
                const int64_t l = i ^ j;
                if (l > i) {
                    const int32_t x = a[i], y = a[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// rows of 33..kMidMax entries: one CTA each, sorted in shared memory
__global__ void sweep_csr_mid_kernel(int n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                     const int32_t *__restrict__ newid, const int32_t *__restrict__ inv,
                                     const int64_t *__restrict__ rp_new, int32_t *__restrict__ col_new) {
    __shared__ int32_t a[kMidMax];
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t d = rp_new[r + 1] - rp_new[r];
        if (d <= 32 || d > kMidMax) continue;
        const int64_t p = next_pow2(d);
        const int64_t src = row_ptr[inv[r]];
        for (int64_t i = threadIdx.x; i < p; i += blockDim.x) a[i] = i < d ? newid[col[src + i]] : INT_MAX;
        __syncthreads();
        cta_bitonic(a, p);
        for (int64_t i = threadIdx.x; i < d; i += blockDim.x) col_new[rp_new[r] + i] = a[i];
        __syncthreads();
    }
}

// rows longer than kMidMax: one CTA each on a padded copy at pad + poff[r]
__global__ void sweep_csr_big_kernel(int n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                     const int32_t *__restrict__ newid, const int32_t *__restrict__ inv,
                                     const int64_t *__restrict__ rp_new, const int64_t *__restrict__ poff,
                                     int32_t *__restrict__ pad, int32_t *__restrict__ col_new) {
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t d = rp_new[r + 1] - rp_new[r];
        if (d <= kMidMax) continue;
        const int64_t p = poff[r + 1] - poff[r];   // next power of two of d
        int32_t *a = pad + poff[r];
        const int64_t src = row_ptr[inv[r]];
        for (int64_t i = threadIdx.x; i < p; i += blockDim.x) a[i] = i < d ? newid[col[src + i]] : INT_MAX;
        __syncthreads();
        cta_bitonic(a, p);
        for (int64_t i = threadIdx.x; i < d; i += blockDim.x) col_new[rp_new[r] + i] = a[i];
        __syncthreads();
    }
}

}  // namespace

size_t sweep_csr_workspace_bytes(int64_t n, int64_t nnz) {
    const int64_t tiles = std::max<int64_t>(1, ceil_div(n + 1, kScanTile));
    return 4 * (((size_t)(n + 1) * 8 + 255) & ~size_t(255))   // deg, padded, rp_new, poff
           + (((size_t)tiles * 8 + 255) & ~size_t(255))        // scan tile sums
           + (((size_t)nnz * 4 + 255) & ~size_t(255))          // col_new
           + (((size_t)nnz * 8 + 255) & ~size_t(255));         // padded copies of the long rows (<= 2 nnz ints)
}

int sweep_csr_relabel_launch(int n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, const SweepBuffers &sb,
                             void *ws, int64_t **rp_new_out, int32_t **col_new_out, int num_sms,
                             cudaStream_t stream) {
    unsigned char *p = static_cast<unsigned char *>(ws);
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += (bytes + 255) & ~size_t(255);
        return q;
    };
    int64_t *deg = reinterpret_cast<int64_t *>(take((size_t)(n + 1) * 8));
    int64_t *padded = reinterpret_cast<int64_t *>(take((size_t)(n + 1) * 8));
    int64_t *rp_new = reinterpret_cast<int64_t *>(take((size_t)(n + 1) * 8));
    int64_t *poff = reinterpret_cast<int64_t *>(take((size_t)(n + 1) * 8));
    int64_t *sums = reinterpret_cast<int64_t *>(take((size_t)std::max<int64_t>(1, ceil_div(n + 1, kScanTile)) * 8));
    int32_t *col_new = reinterpret_cast<int32_t *>(take((size_t)nnz * 4));
    int32_t *pad = reinterpret_cast<int32_t *>(take((size_t)nnz * 8));
    *rp_new_out = rp_new;
    *col_new_out = col_new;
    if (n <= 0) return CG_OK;
    const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms * 4);
    sweep_csr_degrees_kernel<<<blocks, 256, 0, stream>>>(n, row_ptr, sb.inv, deg, padded);
    CG_LAUNCH_CHECK("sweep_csr_degrees_kernel");
    int rc;
    if ((rc = scan_launch(deg, n, rp_new, sums, stream))) return rc;
    if ((rc = scan_launch(padded, n, poff, sums, stream))) return rc;
    sweep_csr_small_kernel<<<num_sms * 8, 256, 0, stream>>>(n, row_ptr, col, sb.newid, sb.inv, rp_new, col_new);
    CG_LAUNCH_CHECK("sweep_csr_small_kernel");
    sweep_csr_mid_kernel<<<num_sms * 4, 256, 0, stream>>>(n, row_ptr, col, sb.newid, sb.inv, rp_new, col_new);
    CG_LAUNCH_CHECK("sweep_csr_mid_kernel");
    sweep_csr_big_kernel<<<num_sms, 1024, 0, stream>>>(n, row_ptr, col, sb.newid, sb.inv, rp_new, poff, pad,
                                                        col_new);
    CG_LAUNCH_CHECK("sweep_csr_big_kernel");
    return CG_OK;
}

}  // namespace cg
