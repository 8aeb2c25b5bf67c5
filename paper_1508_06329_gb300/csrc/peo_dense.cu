// peo_dense.cu — perfect-elimination check of dense graphs (Sections 5.2, 6.2).
//
// For every vertex v (one warp per vertex, all graphs of a batch in one grid):
//   p(v)  = the neighbour of v with the largest order index below pos(v)
//           (the paper's preparationLNandP kernel) — taken from the LexBFS
//           kernel, which records it, or computed here for a given order;
//   bad   = (LN_v - {p}) \ N(p), evaluated word by word as row_v & ~row_p and
//           kept only for bits u != p with pos(u) < pos(v) (the paper's
//           testing kernel, with p itself excluded);
// and the first violation in order is found by an atomicMin over the 64-bit
// key (pos(v) << 32 | u), u being the lowest id of bad(v) (the lane whose word
// holds the lowest violating bit wins the warp min-reduction).
// The finalize kernel turns each graph's key into (chordal, v, p, u).
#include <algorithm>

#include "kernels.h"

namespace cg {

namespace {

constexpr int kPeoThreads = 256;

constexpr int kRC = 16;   // row words per lane held in registers (512 words = 16,384 vertices per chunk)

template <bool PARENT_KNOWN>
__global__ void __launch_bounds__(kPeoThreads) peo_dense_kernel(const DenseDesc *__restrict__ descs,
                                                                DenseDesc single, int count,
                                                                const int64_t *__restrict__ voff, int64_t total,
                                                                const int32_t *__restrict__ order,
                                                                const int32_t *__restrict__ pos,
                                                                int32_t *__restrict__ parent,
                                                                unsigned long long *__restrict__ keys) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t vbase0 = descs ? __ldg(voff) : 0;   // voff may be a slice of a larger offset table
    for (int64_t gr = warp; gr < total; gr += nwarps) {
        const int64_t gv = gr + vbase0;
        int gi = 0;
        if (descs) {
            int lo = 0, hi = count;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(voff + mid) <= gv) lo = mid; else hi = mid;
            }
            gi = lo;
        }
        const DenseDesc d = descs ? descs[gi] : single;
        const int v = (int)(gv - (descs ? __ldg(voff + gi) : 0));
        const int wn = (d.n + 31) >> 5;
        const uint32_t lastmask = (d.n & 31) ? ((1u << (d.n & 31)) - 1u) : 0xFFFFFFFFu;
        const int32_t *pos_g = pos + d.vbase;
        const int pv = __ldg(pos_g + v);
        const uint32_t *rv = d.rows + (size_t)v * d.words;

        int p;
        if (PARENT_KNOWN) {
            p = __ldg(parent + d.vbase + v);
        } else {
            int best = -1;
            for (int w0 = 0; w0 < wn; w0 += 32 * kRC) {
                uint32_t a[kRC];
#pragma unroll
                for (int k = 0; k < kRC; ++k) {
                    const int w = w0 + k * 32 + lane;
                    a[k] = w < wn ? __ldg(rv + w) : 0u;
                    if (w == wn - 1) a[k] &= lastmask;
                }
#pragma unroll
                for (int k = 0; k < kRC; ++k) {
                    uint32_t bits = a[k];
                    const int w = w0 + k * 32 + lane;
                    while (bits) {
                        const int u = (w << 5) + (__ffs(bits) - 1);
                        bits &= bits - 1;
                        const int pu = __ldg(pos_g + u);
                        if (pu < pv && pu > best) best = pu;
                    }
                }
            }
            best = __reduce_max_sync(0xFFFFFFFFu, best);
            p = best >= 0 ? __ldg(order + d.obase + best) : -1;
            if (lane == 0) parent[d.vbase + v] = p;
        }
        if (p < 0) continue;

        // LN_v - {p} ⊆ N(p): scan row_v & ~row_p for an earlier vertex other than p
        const uint32_t *rp = d.rows + (size_t)p * d.words;
        unsigned umin = 0xFFFFFFFFu;
        for (int w0 = 0; w0 < wn && umin == 0xFFFFFFFFu; w0 += 32 * kRC) {
            uint32_t a[kRC], b[kRC];
#pragma unroll
            for (int k = 0; k < kRC; ++k) {
                const int w = w0 + k * 32 + lane;
                a[k] = w < wn ? __ldg(rv + w) : 0u;
                b[k] = w < wn ? __ldg(rp + w) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kRC; ++k) {
                const int w = w0 + k * 32 + lane;
                uint32_t bits = a[k] & ~b[k];
                if (w == wn - 1) bits &= lastmask;
                if (w == (p >> 5)) bits &= ~(1u << (p & 31));
                while (bits && umin == 0xFFFFFFFFu) {
                    const int u = (w << 5) + (__ffs(bits) - 1);
                    bits &= bits - 1;
                    if (__ldg(pos_g + u) < pv) umin = (unsigned)u;
                }
            }
            umin = __reduce_min_sync(0xFFFFFFFFu, umin);
        }
        if (lane == 0 && umin != 0xFFFFFFFFu)
            atomicMin(keys + gi, ((unsigned long long)(unsigned)pv << 32) | umin);
    }
}

__global__ void finalize_kernel(const DenseDesc *__restrict__ descs, DenseDesc single, int count,
                                const unsigned long long *__restrict__ keys, const int32_t *__restrict__ order,
                                const int32_t *__restrict__ parent, cg_result *__restrict__ res) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= count) return;
    const DenseDesc d = descs ? descs[gi] : single;
    const unsigned long long k = keys[gi];
    cg_result r;
    if (k == ~0ull) {
        r.chordal = 1;
        r.v = r.p = r.u = -1;
    } else {
        const int pv = (int)(k >> 32);
        r.chordal = 0;
        r.v = order[d.obase + pv];
        r.p = parent[d.vbase + r.v];
        r.u = (int)(k & 0xFFFFFFFFu);
    }
    res[descs ? d.rindex : gi] = r;
}

__global__ void invert_order_kernel(const DenseDesc *__restrict__ descs, DenseDesc single, int count,
                                    const int64_t *__restrict__ voff, int64_t total,
                                    const int32_t *__restrict__ order, int32_t *__restrict__ pos) {
    const int64_t vbase0 = descs ? __ldg(voff) : 0;
    for (int64_t gr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gr < total;
         gr += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gv = gr + vbase0;
        int gi = 0;
        if (descs) {
            int lo = 0, hi = count;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(voff + mid) <= gv) lo = mid; else hi = mid;
            }
            gi = lo;
        }
        const DenseDesc d = descs ? descs[gi] : single;
        const int i = (int)(gv - (descs ? __ldg(voff + gi) : 0));
        const int x = order[d.obase + i];
        if (x >= 0 && x < d.n) pos[d.vbase + x] = i;
    }
}

}  // namespace

int invert_order_launch(const DenseDesc *descs, DenseDesc single, int count, const int64_t *voff, int64_t total,
                        const int32_t *order, int32_t *pos, int num_sms, cudaStream_t stream) {
    if (total <= 0) return CG_OK;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), (int64_t)num_sms * 8));
    invert_order_kernel<<<blocks, 256, 0, stream>>>(descs, single, count, voff, total, order, pos);
    CG_LAUNCH_CHECK("invert_order_kernel");
    return CG_OK;
}

int peo_dense_launch(const DenseDesc *descs, DenseDesc single, int count, const int64_t *voff, int64_t total,
                     const int32_t *order, const int32_t *pos, int32_t *parent, bool parent_known,
                     unsigned long long *keys, int num_sms, cudaStream_t stream) {
    if (count <= 0) return CG_OK;
    CG_CUDA_TRY(cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * count, stream));
    if (total <= 0) return CG_OK;
    const int64_t warps_needed = total;
    const int64_t blocks_needed = ceil_div(warps_needed, kPeoThreads / 32);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, (int64_t)num_sms * 8));
    if (parent_known)
        peo_dense_kernel<true><<<blocks, kPeoThreads, 0, stream>>>(descs, single, count, voff, total, order, pos,
                                                                   parent, keys);
    else
        peo_dense_kernel<false><<<blocks, kPeoThreads, 0, stream>>>(descs, single, count, voff, total, order, pos,
                                                                    parent, keys);
    CG_LAUNCH_CHECK("peo_dense_kernel");
    return CG_OK;
}

int finalize_launch(const DenseDesc *descs, DenseDesc single, int count, const unsigned long long *keys,
                    const int32_t *order, const int32_t *parent, cg_result *res, cudaStream_t stream) {
    if (count <= 0) return CG_OK;
    finalize_kernel<<<(int)ceil_div(count, 128), 128, 0, stream>>>(descs, single, count, keys, order, parent, res);
    CG_LAUNCH_CHECK("finalize_kernel");
    return CG_OK;
}

}  // namespace cg
