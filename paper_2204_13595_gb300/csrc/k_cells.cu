// k_cells.cu -- wrap/quantise, counting sort into the canonical cell grid.
//
// Sec. 2.3 bins atoms into cells of edge r_eta (here: L/floor(L/r_c)) and
// scans a stencil of cells around each atom.  The sort below orders atoms by
// (cell, caller index) so that every stencil row is a contiguous range of the
// sorted arrays and the shell ordinals of the RBL sampler follow one canonical
// order.  All kernels here are HBM/atomic bound.
#include "rbe_internal.cuh"

namespace {

constexpr int TPB = 256;

// Wrap, quantise, bin; latch non-finite input; per-block sums of q^2, q, |q|.
__global__ void __launch_bounds__(TPB) k_quantize_count(int n, const double* __restrict__ pos,
                                                        const double* __restrict__ q, RbeConsts c,
                                                        int* __restrict__ cell_count, int* __restrict__ cell_of,
                                                        int* __restrict__ slot, double* __restrict__ part_q,
                                                        int* __restrict__ status)
{
    double sq2 = 0.0, sq = 0.0, sabs = 0.0;
    for (int i = blockIdx.x * TPB + threadIdx.x; i < n; i += gridDim.x * TPB) {
        double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        double qi = q[i];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qi)) {
            latch_status(status, RBE_ST_NONFINITE);
            x = y = z = 0.0;
        }
        double xw;
        uint32_t sx, sy, sz;
        wrap_fixed(x, c.invL, c.L, xw, sx);
        wrap_fixed(y, c.invL, c.L, xw, sy);
        wrap_fixed(z, c.invL, c.L, xw, sz);
        uint32_t cx = cell_of_fixed(sx, c.n_cell), cy = cell_of_fixed(sy, c.n_cell), cz = cell_of_fixed(sz, c.n_cell);
        int cell = (int)(cx + (uint32_t)c.n_cell * (cy + (uint32_t)c.n_cell * cz));
        cell_of[i] = cell;
        slot[i] = atomicAdd(&cell_count[cell], 1);
        sq2 += qi * qi;
        sq += qi;
        sabs += fabs(qi);
    }
    __shared__ double red[3][TPB / 32];
    sq2 = warp_sum(sq2); sq = warp_sum(sq); sabs = warp_sum(sabs);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = sq2; red[1][w] = sq; red[2][w] = sabs; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double a = 0.0;
        for (int k = 0; k < TPB / 32; ++k) a += red[threadIdx.x][k];
        part_q[blockIdx.x * RBE_NPART_Q + threadIdx.x] = a;
    }
}

// Exclusive scan of cell_count[0..m) into start[0..m] (single block).
__global__ void __launch_bounds__(1024) k_scan(long m, const int* __restrict__ count, int* __restrict__ start)
{
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int T = 1024;
    long per = (m + (long)T * 4 - 1) / ((long)T * 4);   // elements per thread per pass: 4*per chunks
    // process in passes of T*per elements, each thread a contiguous run
    long chunk = per * 4;
    for (long base = 0; base < m; base += chunk * T) {
        long b = base + (long)threadIdx.x * chunk;
        long e = b + chunk < m ? b + chunk : m;
        int local = 0;
        for (long k = b; k < e; ++k) local += count[k];
        // inclusive warp scan of local sums
        int v = local;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        if (w == 0) {
            int s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        int excl = carry + v - local + (w > 0 ? wsum[w - 1] : 0);
        int run = excl;
        for (long k = b; k < e; ++k) { start[k] = run; run += count[k]; }
        __syncthreads();
        if (threadIdx.x == T - 1) carry = excl + local;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[m] = carry;
}

__global__ void __launch_bounds__(TPB) k_scatter(int n, const int* __restrict__ cell_of, const int* __restrict__ slot,
                                                 const int* __restrict__ start, int* __restrict__ perm)
{
    int i = blockIdx.x * TPB + threadIdx.x;
    if (i < n) perm[start[cell_of[i]] + slot[i]] = i;
}

// Canonical in-cell order: ascending caller index (insertion sort, cells are small).
__global__ void __launch_bounds__(TPB) k_sort_cells(long m, const int* __restrict__ start, int* __restrict__ perm)
{
    long c = (long)blockIdx.x * TPB + threadIdx.x;
    if (c >= m) return;
    int b = start[c], e = start[c + 1];
    for (int k = b + 1; k < e; ++k) {
        int v = perm[k];
        int t = k - 1;
        while (t >= b && perm[t] > v) { perm[t + 1] = perm[t]; --t; }
        perm[t + 1] = v;
    }
}

__global__ void __launch_bounds__(TPB) k_gather(int n, const int* __restrict__ perm, const double* __restrict__ pos,
                                                const double* __restrict__ q, const int32_t* __restrict__ type,
                                                const int32_t* __restrict__ mol, RbeConsts c, uint4* __restrict__ s4,
                                                float4* __restrict__ f4, double4_32a* __restrict__ p4, int2* __restrict__ tm,
                                                int* __restrict__ status)
{
    int k = blockIdx.x * TPB + threadIdx.x;
    if (k >= n) return;
    int i = perm[k];
    double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) x = y = z = 0.0;
    double xw, yw, zw;
    uint32_t sx, sy, sz;
    wrap_fixed(x, c.invL, c.L, xw, sx);
    wrap_fixed(y, c.invL, c.L, yw, sy);
    wrap_fixed(z, c.invL, c.L, zw, sz);
    double qi = q[i];
    float qf = (float)qi;
    s4[k] = make_uint4(sx, sy, sz, __float_as_uint(qf));
    f4[k] = make_float4((float)xw, (float)yw, (float)zw, qf);
    p4[k] = make_double4_32a(xw, yw, zw, qi);
    int t = type ? type[i] : 0;
    if (t < 0 || t >= c.ntypes) {
        latch_status(status, RBE_ST_BADTYPE);
        t = 0;
    }
    tm[k] = make_int2(t, mol ? mol[i] : -(i + 1));
}

}  // namespace

void launch_quantize_count(rbe_ctx* ctx, int n, const double* pos, const double* q, cudaStream_t st)
{
    cudaMemsetAsync(ctx->cell_count, 0, sizeof(int) * (size_t)(ctx->ncells + 1), st);
    prof_begin(ctx, RBE_K_QUANTIZE, st);
    k_quantize_count<<<ctx->grid_q, TPB, 0, st>>>(n, pos, q, ctx->c, ctx->cell_count, ctx->cell_of, ctx->slot,
                                                  ctx->part_q, ctx->status);
    prof_end(ctx, RBE_K_QUANTIZE, st);
}

void launch_scan(rbe_ctx* ctx, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_SCAN, st);
    k_scan<<<1, 1024, 0, st>>>(ctx->ncells, ctx->cell_count, ctx->cell_start);
    prof_end(ctx, RBE_K_SCAN, st);
}

void launch_scatter_sort_gather(rbe_ctx* ctx, int n, const double* pos, const double* q, const int32_t* type,
                                const int32_t* mol, cudaStream_t st)
{
    int g = (n + TPB - 1) / TPB;
    prof_begin(ctx, RBE_K_SCATTER, st);
    k_scatter<<<g, TPB, 0, st>>>(n, ctx->cell_of, ctx->slot, ctx->cell_start, ctx->perm);
    prof_end(ctx, RBE_K_SCATTER, st);
    prof_begin(ctx, RBE_K_SORT, st);
    k_sort_cells<<<(unsigned)((ctx->ncells + TPB - 1) / TPB), TPB, 0, st>>>(ctx->ncells, ctx->cell_start, ctx->perm);
    prof_end(ctx, RBE_K_SORT, st);
    prof_begin(ctx, RBE_K_GATHER, st);
    k_gather<<<g, TPB, 0, st>>>(n, ctx->perm, pos, q, type, mol, ctx->c, ctx->s4, ctx->f4, ctx->p4, ctx->tm,
                                 ctx->status);
    prof_end(ctx, RBE_K_GATHER, st);
}
