// k_rbl.cu -- random batch list (RBL) real-space kernel, Sec. 2.3.
//
// One warp per atom i (sorted order), fused:
//   1. list construction: the warp walks the rows of the cell stencil of
//      Sec. 2.3 (reach floor(r_s/w)+1 cells, w the cell edge) in canonical
//      (ascending cell, atom index) order; each row is one or two contiguous
//      ranges of the cell-sorted arrays, trimmed per atom to the cells that
//      can hold a point within r_s.  Candidates are classified by exact
//      integer squared distance on the fixed-point coordinates into the core
//      C(i) (r <= r_c) and shell S(i) (r_c < r <= r_s) and appended, in
//      order, to per-warp shared-memory buffers (ballot + popc ranks);
//   2. shell batch: if N_S > p, Floyd's algorithm draws p distinct ordinals
//      in [0, N_S) from Philox words at counter (i, k/4, step, 1); otherwise
//      the batch is all of S(i) with weight 1 (Algorithm 1, shell step);
//   3. pair forces f_ij of Eq. (2.10) over C(i) (weight 1) and B(i) (weight
//      N_S/p, Eq. (2.11)); same-molecule pairs take the Ewald exclusion
//      correction instead of erfc + LJ.
// Outputs: F_real (core + weighted shell, before the momentum correction of
// Eq. (2.13)) per sorted atom, and per-block partial sums of the real-space
// energies, the virial and the net force (deterministic fixed-order sums).
#include <math.h>

#include "rbe_internal.cuh"

namespace {

struct RblArgs {
    int n;
    uint64_t step;
    const uint4* __restrict__ s4;
    const double4_32a* __restrict__ p4;
    const int2* __restrict__ tm;
    const int* __restrict__ perm;
    const int* __restrict__ cell_start;
    const RbeLJ* __restrict__ lj;
    double* __restrict__ F_real;
    double* __restrict__ part;
    int* __restrict__ status;
    RbeConsts c;
    int core_cap, shell_cap, p_pad;
    int debug, dbg_cap;
    int* __restrict__ dbg_ncore;
    int* __restrict__ dbg_nshell;
    int* __restrict__ dbg_core;
    int* __restrict__ dbg_batch;
};

// Ascending k-th distinct cell of the stencil along one axis and its offset
// d in [-R, R] from the atom's cell c (ring of nc cells).
__device__ __forceinline__ void axis_cell(int k, int c, int R, int nc, bool full, int& cell, int& off)
{
    if (full) { cell = k; off = 0; return; }
    if (c - R < 0) {
        cell = (k <= c + R) ? k : (c - R + nc + (k - (c + R + 1)));
    } else if (c + R >= nc) {
        cell = (k <= c + R - nc) ? k : (c - R + (k - (c + R - nc + 1)));
    } else {
        cell = c - R + k;
    }
    int d = cell - c;
    if (d > R) d -= nc;
    if (d < -R) d += nc;
    off = d;
}

// Distance (fraction of L) from fractional coordinate f in cell c to the
// slab of the cell at offset d (unwrapped): a lower bound for any atom there.
__device__ __forceinline__ float axis_gap(float f, int c, int d, int nc, bool full)
{
    if (full || d == 0) return 0.0f;
    float g = (d > 0) ? (float)(c + d) / (float)nc - f : f - (float)(c + d + 1) / (float)nc;
    return g > 0.0f ? g : 0.0f;
}

template <bool MIXED>
__global__ void __launch_bounds__(RBE_WARPS_RBL * 32) k_rbl(RblArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const RbeConsts& c = a.c;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;

    // shared layout: LJ tables, then per-warp buffers
    const int nt2 = c.ntypes * c.ntypes;
    double* s_c12 = reinterpret_cast<double*>(smem);
    double* s_c6 = s_c12 + nt2;
    double* s_sh = s_c6 + nt2;
    unsigned char* wbase = smem + sizeof(double) * 3 * ((nt2 + 1) & ~1);
    const size_t wbytes = sizeof(uint64_t) * a.p_pad + sizeof(int) * (a.core_cap + a.shell_cap + a.p_pad);
    uint64_t* words = reinterpret_cast<uint64_t*>(wbase + wbytes * wib);
    int* core_buf = reinterpret_cast<int*>(words + a.p_pad);
    int* shell_buf = core_buf + a.core_cap;
    int* sel = shell_buf + a.shell_cap;
    for (int t = threadIdx.x; t < nt2; t += blockDim.x) {
        int ti = t / c.ntypes, tj = t % c.ntypes;
        s_c12[t] = a.lj->c12[ti * RBE_MAXT + tj];
        s_c6[t] = a.lj->c6[ti * RBE_MAXT + tj];
        s_sh[t] = a.lj->shift[ti * RBE_MAXT + tj];
    }
    __syncthreads();

    const int nc = c.n_cell, R = c.reach;
    const bool full = (2 * R + 1 >= nc);
    const int naxis = full ? nc : 2 * R + 1;
    const int nrows = naxis * naxis;
    const float ncf = (float)nc;

    double acc_e[3] = {0.0, 0.0, 0.0};
    double acc_w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double acc_f[3] = {0.0, 0.0, 0.0};
    const int warps_total = gridDim.x * RBE_WARPS_RBL;

    for (int i = blockIdx.x * RBE_WARPS_RBL + wib; i < a.n; i += warps_total) {
        const uint4 si = a.s4[i];
        const int cx = (int)cell_of_fixed(si.x, nc), cy = (int)cell_of_fixed(si.y, nc), cz = (int)cell_of_fixed(si.z, nc);
        const float fx = (float)si.x * 2.3283064365386963e-10f;
        const float fy = (float)si.y * 2.3283064365386963e-10f;
        const float fz = (float)si.z * 2.3283064365386963e-10f;
        int ncore = 0, nshell = 0;
        bool overlap = false;

        // ---- 1. classify the stencil in canonical order ----------------------
        for (int rb = 0; rb < nrows; rb += 32) {
            int b1 = 0, e1 = 0, b2 = 0, e2 = 0;
            int r = rb + lane;
            if (r < nrows) {
                int az = r / naxis, ay = r % naxis;
                int zc, dz, yc, dy;
                axis_cell(az, cz, R, nc, full, zc, dz);
                axis_cell(ay, cy, R, nc, full, yc, dy);
                float gz = axis_gap(fz, cz, dz, nc, full), gy = axis_gap(fy, cy, dy, nc, full);
                float g2 = gz * gz + gy * gy;
                if (g2 <= c.rs_frac2) {
                    int rowbase = nc * (yc + nc * zc);
                    if (full) {
                        b1 = a.cell_start[rowbase];
                        e1 = a.cell_start[rowbase + nc];
                    } else {
                        float hx = sqrtf(c.rs_frac2 - g2) + 1e-5f;
                        int dlo = (int)floorf((fx - hx) * ncf) - cx;
                        int dhi = (int)floorf((fx + hx) * ncf) - cx;
                        dlo = dlo < -R ? -R : dlo;
                        dhi = dhi > R ? R : dhi;
                        int ca = cx + dlo, cb = cx + dhi;
                        int lo1, hi1, lo2 = 0, hi2 = -1;
                        if (ca < 0) { lo1 = 0; hi1 = cb; lo2 = ca + nc; hi2 = nc - 1; }
                        else if (cb >= nc) { lo1 = 0; hi1 = cb - nc; lo2 = ca; hi2 = nc - 1; }
                        else { lo1 = ca; hi1 = cb; }
                        b1 = a.cell_start[rowbase + lo1];
                        e1 = a.cell_start[rowbase + hi1 + 1];
                        if (hi2 >= lo2) {
                            b2 = a.cell_start[rowbase + lo2];
                            e2 = a.cell_start[rowbase + hi2 + 1];
                        }
                    }
                }
            }
            int rcount = nrows - rb < 32 ? nrows - rb : 32;
            for (int rr = 0; rr < rcount; ++rr) {
                int rb1 = __shfl_sync(FULL, b1, rr), re1 = __shfl_sync(FULL, e1, rr);
                int rb2 = __shfl_sync(FULL, b2, rr), re2 = __shfl_sync(FULL, e2, rr);
#pragma unroll 1
                for (int part = 0; part < 2; ++part) {
                    int beg = part ? rb2 : rb1, end = part ? re2 : re1;
                    for (int base = beg; base < end; base += 32) {
                        int j = base + lane;
                        bool valid = j < end;
                        uint4 sj = valid ? a.s4[j] : si;
                        int ddx = (int)(sj.x - si.x), ddy = (int)(sj.y - si.y), ddz = (int)(sj.z - si.z);
                        unsigned long long d2 = (unsigned long long)((long long)ddx * ddx) +
                                                (unsigned long long)((long long)ddy * ddy) +
                                                (unsigned long long)((long long)ddz * ddz);
                        bool other = valid && j != i;
                        bool is_core = other && d2 <= c.Rc2;
                        bool is_shell = other && d2 > c.Rc2 && d2 <= c.Rs2;
                        overlap |= other && d2 == 0ull;
                        unsigned cm = __ballot_sync(FULL, is_core), sm = __ballot_sync(FULL, is_shell);
                        int cpos = ncore + __popc(cm & lt_mask), spos = nshell + __popc(sm & lt_mask);
                        if (is_core && cpos < a.core_cap) core_buf[cpos] = j;
                        if (is_shell && spos < a.shell_cap) shell_buf[spos] = j;
                        ncore += __popc(cm);
                        nshell += __popc(sm);
                    }
                }
            }
        }
        if (__any_sync(FULL, overlap) && lane == 0) latch_status(a.status, RBE_ST_OVERLAP);
        if ((ncore > a.core_cap || nshell > a.shell_cap) && lane == 0) latch_status(a.status, RBE_ST_CAPACITY);
        const int ncore_c = ncore < a.core_cap ? ncore : a.core_cap;
        const int gi = a.perm[i];

        // ---- 2. shell batch (Floyd over ordinals) ---------------------------
        const int p = c.p;
        const bool sample = nshell > p;
        const int nb = sample ? p : nshell;
        if (sample) {
            for (int b = lane; 4 * b < p; b += 32) {
                uint64_t w[4];
                philox4x64_10((uint64_t)gi, (uint64_t)b, a.step, 1ull, c.seed, 0ull, w);
#pragma unroll
                for (int qd = 0; qd < 4; ++qd) words[4 * b + qd] = w[qd];
            }
            __syncwarp();
            for (int k = 0; k < p; ++k) {
                uint64_t jj = (uint64_t)(nshell - p + k);
                int t = (int)__umul64hi(words[k], jj + 1ull);
                bool dup = false;
                for (int l = lane; l < k; l += 32) dup |= (sel[l] == t);
                dup = __any_sync(FULL, dup);
                if (lane == 0) sel[k] = dup ? (int)jj : t;
                __syncwarp();
            }
        }
        __syncwarp();
        const double wsh = sample ? (double)nshell / (double)p : 1.0;

        // ---- 3. pair terms over C(i) and B(i) -------------------------------
        double fi[3] = {0.0, 0.0, 0.0};
        const int npairs = ncore_c + nb;
        if (MIXED) {
            const float qi = __uint_as_float(si.w);
            const int2 ti = a.tm[i];
            const float kef = (float)c.k_e, saf = (float)c.sqrt_alpha, tsaf = (float)c.two_sqrt_alpha_over_sqrt_pi;
            float ff[3] = {0.f, 0.f, 0.f}, fe[3] = {0.f, 0.f, 0.f}, fw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int t = lane; t < npairs; t += 32) {
                int j;
                float w;
                if (t < ncore_c) { j = core_buf[t]; w = 1.0f; }
                else {
                    int k = t - ncore_c;
                    int ord = sample ? sel[k] : k;
                    ord = ord < a.shell_cap ? ord : a.shell_cap - 1;
                    j = shell_buf[ord];
                    w = (float)wsh;
                }
                const uint4 sj = a.s4[j];
                const int2 tj = a.tm[j];
                float dx = (float)(int)(sj.x - si.x) * c.Lfix;
                float dy = (float)(int)(sj.y - si.y) * c.Lfix;
                float dz = (float)(int)(sj.z - si.z) * c.Lfix;
                float r2 = dx * dx + dy * dy + dz * dz;
                float rinv = rsqrtf(r2);
                float r = r2 * rinv;
                float qq = kef * qi * __uint_as_float(sj.w);
                float ar = saf * r;
                float gauss = tsaf * expf(-ar * ar);
                float s, uc = 0.f, ul = 0.f, ux = 0.f;
                if (ti.y == tj.y) {
                    float er = erff(ar);
                    s = -qq * (gauss * rinv - er * rinv * rinv) * rinv;
                    ux = -qq * er * rinv;
                } else {
                    float ec = erfcf(ar);
                    s = -qq * (ec * rinv * rinv + gauss * rinv) * rinv;
                    uc = qq * ec * rinv;
                    int tt = ti.x * c.ntypes + tj.x;
                    float c12 = (float)s_c12[tt], c6 = (float)s_c6[tt];
                    if (c12 != 0.f || c6 != 0.f) {
                        float ir2 = rinv * rinv;
                        float ir6 = ir2 * ir2 * ir2;
                        s += -(12.f * c12 * ir6 * ir6 - 6.f * c6 * ir6) * ir2;
                        ul = c12 * ir6 * ir6 - c6 * ir6 - (float)s_sh[tt];
                    }
                }
                float gx = w * s * dx, gy = w * s * dy, gz = w * s * dz;
                ff[0] += gx; ff[1] += gy; ff[2] += gz;
                fe[0] += w * uc; fe[1] += w * ul; fe[2] += w * ux;
                fw[0] += dx * gx; fw[1] += dy * gy; fw[2] += dz * gz;
                fw[3] += dx * gy; fw[4] += dx * gz; fw[5] += dy * gz;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) { fi[q] = (double)ff[q]; acc_e[q] += (double)fe[q]; }
#pragma unroll
            for (int q = 0; q < 6; ++q) acc_w[q] += (double)fw[q];
        } else {
            const double4_32a pi = a.p4[i];
            const int2 ti = a.tm[i];
            for (int t = lane; t < npairs; t += 32) {
                int j;
                double w;
                if (t < ncore_c) { j = core_buf[t]; w = 1.0; }
                else {
                    int k = t - ncore_c;
                    int ord = sample ? sel[k] : k;
                    ord = ord < a.shell_cap ? ord : a.shell_cap - 1;
                    j = shell_buf[ord];
                    w = wsh;
                }
                const double4_32a pj = a.p4[j];
                const int2 tj = a.tm[j];
                double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                dx -= c.L * rint(dx * c.invL);
                dy -= c.L * rint(dy * c.invL);
                dz -= c.L * rint(dz * c.invL);
                double r2 = dx * dx + dy * dy + dz * dz;
                double r = sqrt(r2);
                double rinv = 1.0 / r;
                double qq = c.k_e * pi.w * pj.w;
                double ar = c.sqrt_alpha * r;
                double gauss = c.two_sqrt_alpha_over_sqrt_pi * exp(-ar * ar);
                double s, uc = 0.0, ul = 0.0, ux = 0.0;
                if (ti.y == tj.y) {
                    double er = erf(ar);
                    s = -qq * (gauss * rinv - er * rinv * rinv) * rinv;
                    ux = -qq * er * rinv;
                } else {
                    double ec = erfc(ar);
                    s = -qq * (ec * rinv * rinv + gauss * rinv) * rinv;
                    uc = qq * ec * rinv;
                    int tt = ti.x * c.ntypes + tj.x;
                    double c12 = s_c12[tt], c6 = s_c6[tt];
                    if (c12 != 0.0 || c6 != 0.0) {
                        double ir2 = rinv * rinv;
                        double ir6 = ir2 * ir2 * ir2;
                        s += -(12.0 * c12 * ir6 * ir6 - 6.0 * c6 * ir6) * ir2;
                        ul = c12 * ir6 * ir6 - c6 * ir6 - s_sh[tt];
                    }
                }
                double gx = w * s * dx, gy = w * s * dy, gz = w * s * dz;
                fi[0] += gx; fi[1] += gy; fi[2] += gz;
                acc_e[0] += w * uc; acc_e[1] += w * ul; acc_e[2] += w * ux;
                acc_w[0] += dx * gx; acc_w[1] += dy * gy; acc_w[2] += dz * gz;
                acc_w[3] += dx * gy; acc_w[4] += dx * gz; acc_w[5] += dy * gz;
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) fi[q] = warp_sum(fi[q]);
        if (lane == 0) {
            a.F_real[3 * (size_t)i + 0] = fi[0];
            a.F_real[3 * (size_t)i + 1] = fi[1];
            a.F_real[3 * (size_t)i + 2] = fi[2];
            acc_f[0] += fi[0]; acc_f[1] += fi[1]; acc_f[2] += fi[2];
        }

        // ---- debug record (caller index order) ------------------------------
        if (a.debug) {
            if (lane == 0) { a.dbg_ncore[gi] = ncore; a.dbg_nshell[gi] = nshell; }
            for (int t = lane; t < a.dbg_cap; t += 32)
                a.dbg_core[(size_t)gi * a.dbg_cap + t] = t < ncore_c ? a.perm[core_buf[t]] : -1;
            for (int k = lane; k < p; k += 32) {
                int id = -1;
                if (k < nb) {
                    int ord = sample ? sel[k] : k;
                    ord = ord < a.shell_cap ? ord : a.shell_cap - 1;
                    id = a.perm[shell_buf[ord]];
                }
                a.dbg_batch[(size_t)gi * p + k] = id;
            }
        }
        __syncwarp();
    }

    // ---- deterministic block partials ---------------------------------------
    __shared__ double red[RBE_WARPS_RBL][RBE_NPART_RBL];
    double v[RBE_NPART_RBL] = {acc_e[0], acc_e[1], acc_e[2], acc_w[0], acc_w[1], acc_w[2],
                               acc_w[3], acc_w[4], acc_w[5], acc_f[0], acc_f[1], acc_f[2]};
#pragma unroll
    for (int q = 0; q < RBE_NPART_RBL; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0)
        for (int q = 0; q < RBE_NPART_RBL; ++q) red[wib][q] = v[q];
    __syncthreads();
    if (threadIdx.x < RBE_NPART_RBL) {
        double s = 0.0;
        for (int w = 0; w < RBE_WARPS_RBL; ++w) s += red[w][threadIdx.x];
        a.part[blockIdx.x * RBE_NPART_RBL + threadIdx.x] = s;
    }
}

}  // namespace

int rbl_smem_bytes(const rbe_ctx* ctx)
{
    int nt2 = ctx->c.ntypes * ctx->c.ntypes;
    int p_pad = (ctx->c.p + 3) & ~3;
    size_t head = sizeof(double) * 3 * ((nt2 + 1) & ~1);
    size_t wbytes = sizeof(uint64_t) * p_pad + sizeof(int) * (ctx->core_cap + ctx->shell_cap + p_pad);
    return (int)(head + wbytes * RBE_WARPS_RBL);
}

void launch_rbl(rbe_ctx* ctx, int n, uint64_t step, cudaStream_t st)
{
    RblArgs a;
    a.n = n;
    a.step = step;
    a.s4 = ctx->s4; a.p4 = ctx->p4; a.tm = ctx->tm; a.perm = ctx->perm; a.cell_start = ctx->cell_start;
    a.lj = ctx->lj; a.F_real = ctx->F_real; a.part = ctx->part_rbl; a.status = ctx->status;
    a.c = ctx->c;
    a.core_cap = ctx->core_cap; a.shell_cap = ctx->shell_cap; a.p_pad = (ctx->c.p + 3) & ~3;
    a.debug = ctx->debug; a.dbg_cap = ctx->dbg_cap_core;
    a.dbg_ncore = ctx->dbg_ncore; a.dbg_nshell = ctx->dbg_nshell; a.dbg_core = ctx->dbg_core; a.dbg_batch = ctx->dbg_batch;
    int smem = rbl_smem_bytes(ctx);
    prof_begin(ctx, RBE_K_RBL, st);
    if (ctx->precision == RBE_MIXED) {
        cudaFuncSetAttribute(k_rbl<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_rbl<true><<<ctx->grid_rbl, RBE_WARPS_RBL * 32, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(k_rbl<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_rbl<false><<<ctx->grid_rbl, RBE_WARPS_RBL * 32, smem, st>>>(a);
    }
    prof_end(ctx, RBE_K_RBL, st);
}

int rbl_blocks_per_sm(const rbe_ctx* ctx)
{
    int smem = rbl_smem_bytes(ctx);
    int nb = 0;
    if (ctx->precision == RBE_MIXED) {
        cudaFuncSetAttribute(k_rbl<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rbl<true>, RBE_WARPS_RBL * 32, smem);
    } else {
        cudaFuncSetAttribute(k_rbl<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rbl<false>, RBE_WARPS_RBL * 32, smem);
    }
    return nb > 0 ? nb : 1;
}
