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

// Every kernel body below takes its block index and the block count of its
// replica's grid explicitly (bx, nbx), so that the single-system kernel and
// the batched one (one launch over many replicas) run the same code.

// Stand-in position of an atom whose input position is not finite (the step
// is reported as RBE_ENONFINITE and its result is undefined): the i-th point
// of a cubic lattice of about n points filling the box, so that such atoms
// spread over the cells at the system's own density instead of piling into
// one cell, and the rest of the step costs what a normal step costs.
__device__ __forceinline__ void nonfinite_stand_in(int i, int n, double L, double& x, double& y, double& z)
{
    int m = (int)cbrt((double)n);
    while ((long)m * m * m < (long)n) ++m;
    const double a = L / (double)m;
    x = a * ((double)(i % m) + 0.5);
    y = a * ((double)((i / m) % m) + 0.5);
    z = a * ((double)(i / ((long)m * m)) + 0.5);
}

// Wrap, quantise, bin; latch non-finite input and bad types; per-block sums
// of q^2, q, |q|; the atom's records in caller order (codes and FP32 charge,
// wrapped FP64 position and charge, (type, molecule)) for the gather.  The
// inputs are read once, in order: they may lie in pinned host memory.
__device__ __forceinline__ void quantize_count_body(int bx, int nbx, int n, const double* __restrict__ pos,
                                                    const double* __restrict__ q, const int32_t* __restrict__ type,
                                                    const int32_t* __restrict__ mol, const RbeConsts& c,
                                                    int* __restrict__ cell_count, int* __restrict__ cell_of,
                                                    int* __restrict__ slot, uint32_t* __restrict__ sx_of,
                                                    uint4* __restrict__ rec_s4, double4_32a* __restrict__ rec_p4,
                                                    int2* __restrict__ rec_tm, double* __restrict__ part_q,
                                                    int* __restrict__ status)
{
    double sq2 = 0.0, sq = 0.0, sabs = 0.0;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // block-uniform trip count, so that every lane takes part in the warp
    // vote below; lanes of a warp that fall in the same cell share one atomic
    // (the slot order inside a cell is immaterial: the in-cell sort orders
    // the cell by its keys)
    for (int b0 = bx * TPB; b0 < n; b0 += nbx * TPB) {
        const int i = b0 + threadIdx.x;
        const bool ok = i < n;
        int cell = -1;
        if (ok) {
            double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
            double qi = q[i];
            const bool bad_pos = !isfinite(x) || !isfinite(y) || !isfinite(z);
            if (bad_pos || !isfinite(qi)) latch_status(status, RBE_ST_NONFINITE);
            if (bad_pos) nonfinite_stand_in(i, n, c.L, x, y, z);     // the same rule as the gather
            double xw, yw, zw;
            uint32_t sx, sy, sz;
            wrap_fixed(x, c.invL, c.L, xw, sx);
            wrap_fixed(y, c.invL, c.L, yw, sy);
            wrap_fixed(z, c.invL, c.L, zw, sz);
            uint32_t cx = cell_of_fixed(sx, c.n_cell), cy = cell_of_fixed(sy, c.n_cell), cz = cell_of_fixed(sz, c.n_cell);
            cell = (int)(cx + (uint32_t)c.n_cell * (cy + (uint32_t)c.n_cell * cz));
            cell_of[i] = cell;
            sx_of[i] = sx;
            rec_s4[i] = make_uint4(sx, sy, sz, __float_as_uint((float)qi));
            rec_p4[i] = make_double4_32a(xw, yw, zw, qi);
            int t = type ? type[i] : 0;
            if (t < 0 || t >= c.ntypes) {
                latch_status(status, RBE_ST_BADTYPE);
                t = 0;
            }
            rec_tm[i] = make_int2(t, mol ? mol[i] : -(i + 1));
            sq2 += qi * qi;
            sq += qi;
            sabs += fabs(qi);
        }
        const unsigned peers = __match_any_sync(FULL, cell);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (ok && lane == leader) base = atomicAdd(&cell_count[cell], __popc(peers));
        base = __shfl_sync(FULL, base, leader);
        if (ok) slot[i] = base + __popc(peers & ((1u << lane) - 1u));
    }
    __shared__ double red[3][TPB / 32];
    sq2 = warp_sum(sq2); sq = warp_sum(sq); sabs = warp_sum(sabs);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = sq2; red[1][w] = sq; red[2][w] = sabs; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double a = 0.0;
        for (int k = 0; k < TPB / 32; ++k) a += red[threadIdx.x][k];
        part_q[bx * RBE_NPART_Q + threadIdx.x] = a;
    }
}

__global__ void __launch_bounds__(TPB) k_quantize_count(int n, const double* __restrict__ pos,
                                                        const double* __restrict__ q, const int32_t* __restrict__ type,
                                                        const int32_t* __restrict__ mol, RbeConsts c,
                                                        int* __restrict__ cell_count, int* __restrict__ cell_of,
                                                        int* __restrict__ slot, uint32_t* __restrict__ sx_of,
                                                        uint4* __restrict__ rec_s4, double4_32a* __restrict__ rec_p4,
                                                        int2* __restrict__ rec_tm, double* __restrict__ part_q,
                                                        int* __restrict__ status)
{
    quantize_count_body(blockIdx.x, gridDim.x, n, pos, q, type, mol, c, cell_count, cell_of, slot, sx_of, rec_s4,
                        rec_p4, rec_tm, part_q, status);
}

// Exclusive scan of cell_count[0..m) into start[0..m] (single block).
__device__ __forceinline__ void scan_body(long m, const int* __restrict__ count, int* __restrict__ start)
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

__global__ void __launch_bounds__(1024) k_scan(long m, const int* __restrict__ count, int* __restrict__ start)
{
    scan_body(m, count, start);
}

// Three-phase exclusive scan of the cell counts for large grids: tile sums,
// one block scanning the tile sums, then each tile rescanned with its offset.
// SCAN_TILE cells per block of TPB threads, SCAN_ITEMS consecutive cells per
// thread.  Integer arithmetic: the result is the same as the one-block scan.
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = TPB * SCAN_ITEMS;

__device__ __forceinline__ int block_excl_scan(int v, int& total)
{
    __shared__ int wsum[TPB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int k = 0; k < TPB / 32; ++k) {
        const int x = wsum[k];
        if (k < w) before += x;
        all += x;
    }
    __syncthreads();
    total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(TPB) k_scan_tiles(long m, const int* __restrict__ count, int* __restrict__ tile_sum)
{
    const long base = (long)blockIdx.x * SCAN_TILE + (long)threadIdx.x * SCAN_ITEMS;
    int v = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < m) v += count[base + k];
    int total;
    block_excl_scan(v, total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(TPB) k_scan_top(int ntiles, int* __restrict__ tile_sum, long m,
                                                 int* __restrict__ start)
{
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int t0 = 0; t0 < ntiles; t0 += TPB) {
        const int t = t0 + threadIdx.x;
        const int v = t < ntiles ? tile_sum[t] : 0;
        int total;
        const int ex = block_excl_scan(v, total);
        const int c0 = carry;
        if (t < ntiles) tile_sum[t] = c0 + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry = c0 + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[m] = carry;
}

__global__ void __launch_bounds__(TPB) k_scan_apply(long m, const int* __restrict__ count,
                                                   const int* __restrict__ tile_off, int* __restrict__ start)
{
    const long base = (long)blockIdx.x * SCAN_TILE + (long)threadIdx.x * SCAN_ITEMS;
    int c[SCAN_ITEMS];
    int v = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        c[k] = base + k < m ? count[base + k] : 0;
        v += c[k];
    }
    int total;
    int run = tile_off[blockIdx.x] + block_excl_scan(v, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < m) start[base + k] = run;
        run += c[k];
    }
}

// Scatter into the cell ranges the in-cell sort key (fixed-point x << 32 |
// caller index) of every atom.
__device__ __forceinline__ void scatter_body(int bx, int n, const int* __restrict__ cell_of,
                                             const int* __restrict__ slot, const uint32_t* __restrict__ sx_of,
                                             const int* __restrict__ start, unsigned long long* __restrict__ skey)
{
    int i = bx * TPB + threadIdx.x;
    if (i < n) skey[start[cell_of[i]] + slot[i]] = ((unsigned long long)sx_of[i] << 32) | (unsigned)i;
}

__global__ void __launch_bounds__(TPB) k_scatter(int n, const int* __restrict__ cell_of, const int* __restrict__ slot,
                                                 const uint32_t* __restrict__ sx_of, const int* __restrict__ start,
                                                 unsigned long long* __restrict__ skey)
{
    scatter_body(blockIdx.x, n, cell_of, slot, sx_of, start, skey);
}

// Canonical in-cell order: ascending (fixed-point x code, caller index).
// Sorting by x lets the pair kernel drop, by binary search, the atoms of a
// stencil row's end cells that lie beyond r_s along x.  A warp per cell (cells
// taken warp-strided): the keys are distinct (the caller index is in the low
// word), so each key's place is the number of smaller keys of its cell,
// counted over the warp by shuffles (cells of more than 32 atoms count from
// memory).
__device__ __forceinline__ void sort_cells_body(int bx, int nbx, long m, const int* __restrict__ start,
                                                const unsigned long long* __restrict__ skey, int* __restrict__ perm)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long nw = (long)nbx * (TPB / 32);
    for (long c = (long)bx * (TPB / 32) + (threadIdx.x >> 5); c < m; c += nw) {
        const int b = start[c], cnt = start[c + 1] - b;
        if (cnt <= 32) {
            const unsigned long long key = lane < cnt ? skey[b + lane] : ~0ull;
            int rank = 0;
            for (int k = 0; k < cnt; ++k) rank += __shfl_sync(FULL, key, k) < key ? 1 : 0;
            if (lane < cnt) perm[b + rank] = (int)(unsigned)(key & 0xffffffffull);
        } else {
            for (int t = lane; t < cnt; t += 32) {
                const unsigned long long key = skey[b + t];
                int rank = 0;
                for (int k = 0; k < cnt; ++k) rank += skey[b + k] < key ? 1 : 0;
                perm[b + rank] = (int)(unsigned)(key & 0xffffffffull);
            }
        }
    }
}

__global__ void __launch_bounds__(TPB) k_sort_cells(long m, const int* __restrict__ start,
                                                    const unsigned long long* __restrict__ skey, int* __restrict__ perm)
{
    sort_cells_body(blockIdx.x, gridDim.x, m, start, skey, perm);
}

// Sorted arrays from the quantisation's records: s4 (codes, FP32 charge), f4
// (FP32 wrapped position, charge), p4 (FP64 wrapped position, charge) and tm
// (type, molecule) of sorted atom k = caller atom perm[k].
__device__ __forceinline__ void gather_body(int bx, int n, const int* __restrict__ perm,
                                            const uint4* __restrict__ rec_s4, const double4_32a* __restrict__ rec_p4,
                                            const int2* __restrict__ rec_tm, uint4* __restrict__ s4,
                                            float4* __restrict__ f4, double4_32a* __restrict__ p4,
                                            int2* __restrict__ tm)
{
    int k = bx * TPB + threadIdx.x;
    if (k >= n) return;
    const int i = perm[k];
    const uint4 s = rec_s4[i];
    const double4_32a p = rec_p4[i];
    s4[k] = s;
    f4[k] = make_float4((float)p.x, (float)p.y, (float)p.z, __uint_as_float(s.w));
    p4[k] = p;
    tm[k] = rec_tm[i];
}

__global__ void __launch_bounds__(TPB) k_gather(int n, const int* __restrict__ perm, const uint4* __restrict__ rec_s4,
                                                const double4_32a* __restrict__ rec_p4, const int2* __restrict__ rec_tm,
                                                uint4* __restrict__ s4, float4* __restrict__ f4,
                                                double4_32a* __restrict__ p4, int2* __restrict__ tm)
{
    gather_body(blockIdx.x, n, perm, rec_s4, rec_p4, rec_tm, s4, f4, p4, tm);
}

// ---- Verlet-skin variant: steps between rebuilds -------------------------
// Between rebuilds the sorted order of the last rebuild is kept: every atom
// is wrapped, quantised and written to its slot inv_perm[i] of that order
// (the arrays of gather_body), no counting sort.  The same block sums of q^2,
// q, |q| as quantize_count_body (same grid and loop, so the same rounding).
// An atom whose fixed-point displacement since the rebuild codes sb exceeds
// D2 (skin/2 squared, fixed-point units) sets *moved: a rebuild is due.
__global__ void __launch_bounds__(TPB) k_skin_gather(int n, const double* __restrict__ pos,
                                                     const double* __restrict__ q, const int32_t* __restrict__ type,
                                                     const int32_t* __restrict__ mol, RbeConsts c,
                                                     const int* __restrict__ inv_perm, const uint4* __restrict__ sb,
                                                     uint64_t D2, uint4* __restrict__ s4, float4* __restrict__ f4,
                                                     double4_32a* __restrict__ p4, int2* __restrict__ tm,
                                                     double* __restrict__ part_q, int* __restrict__ status,
                                                     int* __restrict__ moved)
{
    double sq2 = 0.0, sq = 0.0, sabs = 0.0;
    bool far = false;
    for (int b0 = blockIdx.x * TPB; b0 < n; b0 += gridDim.x * TPB) {
        const int i = b0 + threadIdx.x;
        if (i >= n) continue;
        double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        const double qi = q[i];
        const bool bad_pos = !isfinite(x) || !isfinite(y) || !isfinite(z);
        if (bad_pos || !isfinite(qi)) latch_status(status, RBE_ST_NONFINITE);
        if (bad_pos) nonfinite_stand_in(i, n, c.L, x, y, z);
        double xw, yw, zw;
        uint32_t sx, sy, sz;
        wrap_fixed(x, c.invL, c.L, xw, sx);
        wrap_fixed(y, c.invL, c.L, yw, sy);
        wrap_fixed(z, c.invL, c.L, zw, sz);
        const int k = inv_perm[i];
        const uint4 b = sb[k];
        const int dx = (int)(sx - b.x), dy = (int)(sy - b.y), dz = (int)(sz - b.z);
        const unsigned long long d2 = (unsigned long long)((long long)dx * dx) +
                                      (unsigned long long)((long long)dy * dy) +
                                      (unsigned long long)((long long)dz * dz);
        far |= d2 > D2;
        const float qf = (float)qi;
        s4[k] = make_uint4(sx, sy, sz, __float_as_uint(qf));
        f4[k] = make_float4((float)xw, (float)yw, (float)zw, qf);
        p4[k] = make_double4_32a(xw, yw, zw, qi);
        int t = type ? type[i] : 0;
        if (t < 0 || t >= c.ntypes) {
            latch_status(status, RBE_ST_BADTYPE);
            t = 0;
        }
        tm[k] = make_int2(t, mol ? mol[i] : -(i + 1));
        sq2 += qi * qi;
        sq += qi;
        sabs += fabs(qi);
    }
    if (__any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) *moved = 1;
    __shared__ double red[3][TPB / 32];
    sq2 = warp_sum(sq2); sq = warp_sum(sq); sabs = warp_sum(sabs);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = sq2; red[1][w] = sq; red[2][w] = sabs; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double acc = 0.0;
        for (int kk = 0; kk < TPB / 32; ++kk) acc += red[threadIdx.x][kk];
        part_q[blockIdx.x * RBE_NPART_Q + threadIdx.x] = acc;
    }
}

// At a rebuild: the inverse of the new sorted order and the fixed-point codes
// the displacements of later steps are measured from.
__global__ void __launch_bounds__(TPB) k_skin_mark(int n, const int* __restrict__ perm, const uint4* __restrict__ s4,
                                                   int* __restrict__ inv_perm, uint4* __restrict__ sb)
{
    const int k = blockIdx.x * TPB + threadIdx.x;
    if (k >= n) return;
    inv_perm[perm[k]] = k;
    sb[k] = s4[k];
}

// ---- batched forms: one launch over all replicas of a plan -----------------
// Block grids per replica: BK_CELLS = ceil((ncells + 1) / TPB), BK_ATOMS =
// ceil(n / TPB), BK_Q = grid_q, BK_REP = 1.

__global__ void __launch_bounds__(TPB) k_zero_counts_b(const RepDev* __restrict__ R, const int* __restrict__ off,
                                                       int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    long c = (long)bx * TPB + threadIdx.x;
    if (c <= d.ncells) d.cell_count[c] = 0;
}

__global__ void __launch_bounds__(TPB) k_quantize_count_b(const RepDev* __restrict__ R, const int* __restrict__ off,
                                                          int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    quantize_count_body(bx, nbx, d.n, d.pos, d.q, d.type, d.mol, d.c, d.cell_count, d.cell_of, d.slot, d.sx_of,
                        d.rec_s4, d.rec_p4, d.rec_tm, d.part_q, d.status);
}

__global__ void __launch_bounds__(1024) k_scan_b(const RepDev* __restrict__ R)
{
    const RepDev& d = R[blockIdx.x];
    scan_body(d.ncells, d.cell_count, d.cell_start);
}

__global__ void __launch_bounds__(TPB) k_scatter_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    scatter_body(bx, d.n, d.cell_of, d.slot, d.sx_of, d.cell_start, d.skey);
}

__global__ void __launch_bounds__(TPB) k_sort_cells_b(const RepDev* __restrict__ R, const int* __restrict__ off,
                                                      int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    sort_cells_body(bx, nbx, d.ncells, d.cell_start, d.skey, d.perm);
}

__global__ void __launch_bounds__(TPB) k_gather_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    gather_body(bx, d.n, d.perm, d.rec_s4, d.rec_p4, d.rec_tm, d.s4, d.f4, d.p4, d.tm);
}

}  // namespace

void launch_skin_gather(rbe_ctx* ctx, int n, const double* pos, const double* q, const int32_t* type,
                        const int32_t* mol, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_SKIN, st);
    k_skin_gather<<<ctx->grid_q, TPB, 0, st>>>(n, pos, q, type, mol, ctx->c, ctx->inv_perm, ctx->sb, ctx->skin_D2,
                                               ctx->s4, ctx->f4, ctx->p4, ctx->tm, ctx->part_q, ctx->status,
                                               ctx->skin_moved);
    prof_end(ctx, RBE_K_SKIN, st);
}

void launch_skin_mark(rbe_ctx* ctx, int n, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_SKIN, st);
    k_skin_mark<<<(n + TPB - 1) / TPB, TPB, 0, st>>>(n, ctx->perm, ctx->s4, ctx->inv_perm, ctx->sb);
    prof_end(ctx, RBE_K_SKIN, st);
}

void launch_quantize_count(rbe_ctx* ctx, int n, const double* pos, const double* q, const int32_t* type,
                           const int32_t* mol, cudaStream_t st)
{
    cudaMemsetAsync(ctx->cell_count, 0, sizeof(int) * (size_t)(ctx->ncells + 1), st);
    prof_begin(ctx, RBE_K_QUANTIZE, st);
    k_quantize_count<<<ctx->grid_q, TPB, 0, st>>>(n, pos, q, type, mol, ctx->c, ctx->cell_count, ctx->cell_of,
                                                  ctx->slot, ctx->sx_of, ctx->rec_s4, ctx->rec_p4, ctx->rec_tm,
                                                  ctx->part_q, ctx->status);
    prof_end(ctx, RBE_K_QUANTIZE, st);
}

void launch_scan(rbe_ctx* ctx, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_SCAN, st);
    const long m = ctx->ncells;
    const long ntiles = (m + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles <= 2 || !ctx->scan_tmp) {
        k_scan<<<1, 1024, 0, st>>>(m, ctx->cell_count, ctx->cell_start);
    } else {
        k_scan_tiles<<<(unsigned)ntiles, TPB, 0, st>>>(m, ctx->cell_count, ctx->scan_tmp);
        k_scan_top<<<1, TPB, 0, st>>>((int)ntiles, ctx->scan_tmp, m, ctx->cell_start);
        k_scan_apply<<<(unsigned)ntiles, TPB, 0, st>>>(m, ctx->cell_count, ctx->scan_tmp, ctx->cell_start);
    }
    prof_end(ctx, RBE_K_SCAN, st);
}

long scan_tiles(long ncells) { return (ncells + SCAN_TILE - 1) / SCAN_TILE; }

void launch_scatter_sort_gather(rbe_ctx* ctx, int n, cudaStream_t st)
{
    int g = (n + TPB - 1) / TPB;
    prof_begin(ctx, RBE_K_SCATTER, st);
    k_scatter<<<g, TPB, 0, st>>>(n, ctx->cell_of, ctx->slot, ctx->sx_of, ctx->cell_start, ctx->skey);
    prof_end(ctx, RBE_K_SCATTER, st);
    prof_begin(ctx, RBE_K_SORT, st);
    const long wpb = TPB / 32;        // a warp per cell
    k_sort_cells<<<(unsigned)((ctx->ncells + wpb - 1) / wpb), TPB, 0, st>>>(ctx->ncells, ctx->cell_start, ctx->skey,
                                                                            ctx->perm);
    prof_end(ctx, RBE_K_SORT, st);
    prof_begin(ctx, RBE_K_GATHER, st);
    k_gather<<<g, TPB, 0, st>>>(n, ctx->perm, ctx->rec_s4, ctx->rec_p4, ctx->rec_tm, ctx->s4, ctx->f4, ctx->p4,
                                 ctx->tm);
    prof_end(ctx, RBE_K_GATHER, st);
}

void launch_cells_batch(const BatchPlan& bp, cudaStream_t st)
{
    const int nr = bp.nrep;
    k_zero_counts_b<<<bp.total[BK_CELLS], TPB, 0, st>>>(bp.rep, bp.off[BK_CELLS], nr);
    k_quantize_count_b<<<bp.total[BK_Q], TPB, 0, st>>>(bp.rep, bp.off[BK_Q], nr);
    k_scan_b<<<nr, 1024, 0, st>>>(bp.rep);
    k_scatter_b<<<bp.total[BK_ATOMS], TPB, 0, st>>>(bp.rep, bp.off[BK_ATOMS], nr);
    k_sort_cells_b<<<bp.total[BK_CELLS], TPB, 0, st>>>(bp.rep, bp.off[BK_CELLS], nr);
    k_gather_b<<<bp.total[BK_ATOMS], TPB, 0, st>>>(bp.rep, bp.off[BK_ATOMS], nr);
}
