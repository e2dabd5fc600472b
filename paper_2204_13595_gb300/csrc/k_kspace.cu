// k_kspace.cu -- random batch Ewald (RBE) Fourier part, Sec. 2.2, plus the
// deterministic finalisation of the step, bonded water terms and the
// velocity-Verlet kernels.
//
//   k_sample   : P wave vectors from P_k of Eq. (2.8): per axis an exact
//                inverse-CDF draw of the discrete Gaussian
//                exp(-pi^2 m^2/(alpha L^2)) on 64-bit thresholds, (0,0,0)
//                redrawn; Philox counter (l, attempt, step, 2).
//   k_rho      : rho(k_l) = sum_j q_j exp(i k_l.r_j) (Eq. (2.4)); a block owns
//                a contiguous chunk of atoms staged tile by tile in shared
//                memory, each thread owns one k_l and keeps its partial sum in
//                registers; block partials are summed over blocks in a fixed
//                order by k_rho_sum (the single-GPU form of the paper's one
//                MPI_Allreduce of rho(k), Sec. 3).
//   k_kforce   : F_i^{long,*} of Eq. (2.9) with the sampled k_l and rho_l
//                staged in shared memory, combined with the real-space
//                estimate and the momentum correction of Eq. (2.13), written
//                back in the caller's atom order.
// Mixed precision: the phase m.s of the fixed-point coordinates is reduced
// exactly in 32-bit integer arithmetic (k.r = 2 pi (m.s)/2^32 mod 2 pi), then
// evaluated with FP32 sincos; sums go to FP64 every tile.
#include <math.h>

#include "rbe_internal.cuh"

namespace {

constexpr int TILE = 256;
constexpr int TPB = 256;
constexpr int FIN_TPB = 256;   // threads of the batched finalisation block (one replica each)

__device__ __forceinline__ int inv_cdf(uint64_t u, const uint64_t* __restrict__ T, int M)
{
    int lo = 0, hi = 2 * M;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (u < T[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo - M;
}

// Kernel bodies take their block index and their replica's block count
// explicitly (bx, nbx) so that the single-system kernels and the batched ones
// (one launch over many replicas, at the end of this file) share them.
__device__ __forceinline__ void sample_body(int bx, int nbx, const RbeConsts& c, uint64_t step,
                                            const uint64_t* __restrict__ T, const int4* __restrict__ pool,
                                            int4* __restrict__ km, double4_32a* __restrict__ kv,
                                            int* __restrict__ status)
{
    const double twopi_L = 2.0 * 3.14159265358979323846 / c.L;
    for (int l = bx * TPB + threadIdx.x; l < c.P; l += nbx * TPB) {
        int mx = 1, my = 0, mz = 0;
        bool ok = false;
        if (c.kpool > 0) {
            // Algorithm 1: sample l of the step is pool entry floor(u K / 2^64),
            // u word 0 of the block at counter (l, 0, step, 5)
            uint64_t w[4];
            philox4x64_10((uint64_t)l, 0ull, step, 5ull, c.seed, 0ull, w);
            const int4 e = pool[uniform_below(w[0], (uint32_t)c.kpool)];
            mx = e.x; my = e.y; mz = e.z;
            ok = true;
        }
        for (uint64_t t = 0; t < 1024 && !ok; ++t) {
            uint64_t w[4];
            philox4x64_10((uint64_t)l, t, step, 2ull, c.seed, 0ull, w);
            int ax = inv_cdf(w[0], T, c.M), ay = inv_cdf(w[1], T, c.M), az = inv_cdf(w[2], T, c.M);
            if (ax != 0 || ay != 0 || az != 0) { mx = ax; my = ay; mz = az; ok = true; }
        }
        if (!ok) latch_status(status, RBE_ST_KSAMPLE);
        double kx = twopi_L * mx, ky = twopi_L * my, kz = twopi_L * mz;
        double k2 = kx * kx + ky * ky + kz * kz;
        km[l] = make_int4(mx, my, mz, 0);
        kv[l] = make_double4_32a(kx, ky, kz, c.kcoef / k2);
    }
}

__global__ void __launch_bounds__(TPB) k_sample(RbeConsts c, uint64_t step, const uint64_t* __restrict__ T,
                                                const int4* __restrict__ pool, int4* __restrict__ km,
                                                double4_32a* __restrict__ kv, int* __restrict__ status)
{
    sample_body(blockIdx.x, gridDim.x, c, step, T, pool, km, kv, status);
}

// Metropolis-Hastings pool of k samples (Algorithm 1, pool step; Sec. 2.2):
// per axis an independence chain with target w_m (the discrete Gaussian of
// Eq. (2.8)) and proposal q_m = P(round(X) = m), X ~ N(0, alpha L^2/(2 pi^2)),
// both tabulated on the host for |m| <= M; the proposal is drawn by inverse CDF
// on the thresholds Tq, the move m -> m* accepted when
// u < (w_m* q_m) / (w_m q_m*), u = (word >> 11) 2^-53.  Iteration t of axis a
// uses the block at counter (t, a, 0, 4) (word 0 proposal, word 1 acceptance).
// The chains start at 0; after `burn` iterations each iteration emits
// (m_x, m_y, m_z) unless it is 0, until K samples.  One thread: a Markov
// chain is sequential, and the pool is built once per context.
__global__ void k_kpool_build(uint64_t seed, int M, int K, int burn, const double* __restrict__ w,
                              const double* __restrict__ q, const uint64_t* __restrict__ Tq, int4* __restrict__ pool,
                              int* __restrict__ status)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int m[3] = {0, 0, 0};
    int k = 0;
    // bounded: far more iterations than K non-zero samples can need
    const uint64_t tmax = (uint64_t)burn + 64ull * (uint64_t)K + 4096ull;
    for (uint64_t t = 0; k < K; ++t) {
        if (t >= tmax) {
            latch_status(status, RBE_ST_KSAMPLE);
            break;
        }
        for (int a = 0; a < 3; ++a) {
            uint64_t blk[4];
            philox4x64_10(t, (uint64_t)a, 0ull, 4ull, seed, 0ull, blk);
            const int mp = inv_cdf(blk[0], Tq, M);
            const double u = __dmul_rn((double)(blk[1] >> 11), 1.1102230246251565e-16);
            const double r = __ddiv_rn(__dmul_rn(w[mp + M], q[m[a] + M]), __dmul_rn(w[m[a] + M], q[mp + M]));
            if (u < r) m[a] = mp;
        }
        if (t < (uint64_t)burn) continue;
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) continue;
        pool[k++] = make_int4(m[0], m[1], m[2], 0);
    }
}

// FP64 phase factor e^{i theta}, theta = k . x, from the exact 32-bit phase
// ph = m . s mod 2^32 of the fixed-point coordinates (theta = 2 pi ph / 2^32
// + k . delta, delta = x - s L / 2^32 the sub-quantum residual of the
// position, |delta| < L 2^-32): a table of e^{2 pi i j / 65536} for the top
// 16 bits of ph times a Taylor polynomial of the rest, |x| < 2 pi / 65536 +
// |k| |delta| < 1e-4 (cos to x^2, sin to x^3: the first omitted terms are
// below 5e-18).  A fraction of the FP64 work of a general sincos.
__device__ __forceinline__ void cis_fp64(uint32_t ph, double dk, const double2* __restrict__ tab, double& cs,
                                         double& sn)
{
    const double2 e = __ldg(tab + (ph >> 16));
    const double x = fma((double)(ph & 0xFFFFu), 6.283185307179586 * 2.3283064365386963e-10, dk);
    const double x2 = x * x;
    const double c = fma(x2, -0.5, 1.0);
    const double sx = fma(x * x2, -1.0 / 6.0, x);
    cs = e.x * c - e.y * sx;
    sn = e.y * c + e.x * sx;
}

// 64-bit fixed-point code floor(f 2^64) of a fraction 0 <= f < 1, from its
// bits: f 2^64 = significand 2^(e + 12) for the exponent e <= -1 (exact; a
// fraction below 2^-12 loses only bits below 2^-64, and 0 or a subnormal
// gives 0).
__device__ __forceinline__ uint64_t code64(double f)
{
    const uint64_t u = (uint64_t)__double_as_longlong(f);
    const int e = (int)((u >> 52) & 0x7FFull) - 1023;
    const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e + 12;
    return sh >= 0 ? (m << sh) : (-sh < 64 ? (m >> -sh) : 0ull);
}

// The 64-bit code of a wrapped FP64 coordinate 0 <= xw < L (the fraction
// xw / L, taken as xw * (1/L) and folded to [0, 1))
__device__ __forceinline__ uint64_t code64_of(double xw, double invL)
{
    double f = xw * invL;
    if (f >= 1.0) f -= 1.0;
    return code64(f);
}

// FP64 e^{i theta} for theta = 2 pi ph / 2^64 (ph = m . S mod 2^64 of the
// 64-bit codes, exact in integer arithmetic): the table entry of the top 16
// bits times a Taylor polynomial of the remaining 48 bits' angle, |x| <
// 2 pi / 65536 (cos to x^2, sin to x^3: the first omitted terms are below
// 4e-18).  No residual correction: the phase is exact to 2^-64 of a turn.
// (The 1 MB table is read from L2: it costs less than the two FP64
// operations per phase that a 4,096-entry table's longer series took.)
__device__ __forceinline__ void cis_fp64_64(uint64_t ph, const double2* __restrict__ tab, double& cs, double& sn)
{
    const double2 e = __ldg(tab + (ph >> 48));
    const double x = (double)(ph & 0xFFFFFFFFFFFFull) * 3.4061215800865545e-19;     // 2 pi / 2^64
    const double x2 = x * x;
    const double c = fma(x2, -0.5, 1.0);
    const double sx = fma(x * x2, -1.0 / 6.0, x);
    cs = e.x * c - e.y * sx;
    sn = e.y * c + e.x * sx;
}

// Residual delta = x - s L 2^-32 of a wrapped FP64 coordinate and its code.
__device__ __forceinline__ double fixed_residual(double xw, uint32_t s, double Lq)
{
    return fma(-(double)s, Lq, xw);
}

// rho partial sums: block b owns atoms [b*chunk, min(n,(b+1)*chunk)).
template <bool MIXED>
__device__ __forceinline__ void rho_body(int bx, int n, int chunk, const RbeConsts& c, const uint4* __restrict__ s4,
                                         const double4_32a* __restrict__ p4, const int4* __restrict__ km,
                                         const double4_32a* __restrict__ kv, const double2* __restrict__ cis,
                                         double2* __restrict__ part)
{
    __shared__ double4_32a tile_d[MIXED ? 1 : TILE];     // FP64: 64-bit codes (bit patterns) and q
    __shared__ uint4 tile_u[MIXED ? TILE : 1];           // mixed: 32-bit codes and FP32 q
    const int b0 = bx * chunk;
    const int b1 = min(n, b0 + chunk);
    for (int l0 = 0; l0 < c.P; l0 += blockDim.x) {
        const int l = l0 + threadIdx.x;
        const bool act = l < c.P;
        int4 m = act ? km[l] : make_int4(0, 0, 0, 0);
        double re = 0.0, im = 0.0;
        for (int t0 = b0; t0 < b1; t0 += TILE) {
            const int cnt = min(TILE, b1 - t0);
            __syncthreads();
            for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
                if (MIXED) {
                    tile_u[k] = s4[t0 + k];
                } else {
                    // the 64-bit codes (as bit patterns) and the charge
                    const double4_32a p = p4[t0 + k];
                    tile_d[k] = make_double4_32a(__longlong_as_double((long long)code64_of(p.x, c.invL)),
                                                 __longlong_as_double((long long)code64_of(p.y, c.invL)),
                                                 __longlong_as_double((long long)code64_of(p.z, c.invL)), p.w);
                }
            }
            __syncthreads();
            if (act) {
                if (MIXED) {
                    float fre = 0.f, fim = 0.f;
                    const uint32_t mx = (uint32_t)m.x, my = (uint32_t)m.y, mz = (uint32_t)m.z;
                    for (int k = 0; k < cnt; ++k) {
                        uint4 s = tile_u[k];
                        uint32_t ph = mx * s.x + my * s.y + mz * s.z;
                        float ang = (float)(int)ph * 1.4629180792671596e-09f;   // 2 pi / 2^32
                        float sn, cs;
                        __sincosf(ang, &sn, &cs);
                        float q = __uint_as_float(s.w);
                        fre += q * cs;
                        fim += q * sn;
                    }
                    re += (double)fre;
                    im += (double)fim;
                } else {
                    const uint64_t mx = (uint64_t)(long long)m.x, my = (uint64_t)(long long)m.y,
                                   mz = (uint64_t)(long long)m.z;
                    for (int k = 0; k < cnt; ++k) {
                        const double4_32a d = tile_d[k];
                        const uint64_t ph = mx * (uint64_t)__double_as_longlong(d.x) +
                                            my * (uint64_t)__double_as_longlong(d.y) +
                                            mz * (uint64_t)__double_as_longlong(d.z);
                        double sn, cs;
                        cis_fp64_64(ph, cis, cs, sn);
                        re += d.w * cs;
                        im += d.w * sn;
                    }
                }
            }
        }
        if (act) part[(size_t)bx * c.P + l] = make_double2(re, im);
    }
}

template <bool MIXED>
__global__ void k_rho(int n, int chunk, RbeConsts c, const uint4* __restrict__ s4, const double4_32a* __restrict__ p4,
                      const int4* __restrict__ km, const double4_32a* __restrict__ kv, const double2* __restrict__ cis,
                      double2* __restrict__ part)
{
    rho_body<MIXED>(blockIdx.x, n, chunk, c, s4, p4, km, kv, cis, part);
}

// Table of e^{2 pi i j / 65536}, j = 0..65535 (cos, sin), for cis_fp64 and cis_fp64_64.
__global__ void k_cis_table(double2* __restrict__ tab)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 65536) return;
    double sn, cs;
    sincospi((double)j / 32768.0, &sn, &cs);
    tab[j] = make_double2(cs, sn);
}

// Fixed-order sum over blocks; per-k energy and virial terms of the
// reweighted reciprocal sum (E_k = sum_l c_l/2 |rho_l|^2).
// One warp per k: lane t sums the partials of blocks t, t + 32, ... in order,
// then a fixed butterfly; lane 0's result is used (a fixed order).
__device__ __forceinline__ void rho_sum_body(int bx, int nblk, const RbeConsts& c, const double2* __restrict__ part,
                                             const double4_32a* __restrict__ kv, double2* __restrict__ rho,
                                             double* __restrict__ kterms)
{
    const int lane = threadIdx.x & 31;
    const int l = bx * (TPB / 32) + (threadIdx.x >> 5);
    if (l >= c.P) return;
    double re = 0.0, im = 0.0;
#pragma unroll 8
    for (int b = lane; b < nblk; b += 32) {     // (unrolled: several partials' loads in flight)
        double2 v = part[(size_t)b * c.P + l];
        re += v.x;
        im += v.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane != 0) return;
    rho[l] = make_double2(re, im);
    double4_32a k = kv[l];
    double k2 = k.x * k.x + k.y * k.y + k.z * k.z;
    double e = 0.5 * k.w * (re * re + im * im);
    double bb = 2.0 * (1.0 / k2 + 1.0 / (4.0 * c.alpha));
    double* o = kterms + 7 * (size_t)l;
    o[0] = e;
    o[1] = e * (1.0 - bb * k.x * k.x);
    o[2] = e * (1.0 - bb * k.y * k.y);
    o[3] = e * (1.0 - bb * k.z * k.z);
    o[4] = e * (-bb * k.x * k.y);
    o[5] = e * (-bb * k.x * k.z);
    o[6] = e * (-bb * k.y * k.z);
}

__global__ void __launch_bounds__(TPB) k_rho_sum(int nblk, RbeConsts c, const double2* __restrict__ part,
                                                 const double4_32a* __restrict__ kv, double2* __restrict__ rho,
                                                 double* __restrict__ kterms)
{
    rho_sum_body(blockIdx.x, nblk, c, part, kv, rho, kterms);
}

// Harmonic water: molecule m = atoms (3m, 3m+1, 3m+2) = (O, H, H).
__device__ __forceinline__ void bonded_body(int bx, int nbx, int nmol, const double* __restrict__ pos,
                                            const RbeConsts& c, double kb, double r0, double kth, double th0,
                                            double* __restrict__ Fb, double* __restrict__ part)
{
    double u = 0.0;
    for (int mI = bx * TPB + threadIdx.x; mI < nmol; mI += nbx * TPB) {
        int o = 3 * mI;
        double d1[3], d2[3];
        for (int a = 0; a < 3; ++a) {
            double x1 = pos[3 * (o + 1) + a] - pos[3 * o + a];
            double x2 = pos[3 * (o + 2) + a] - pos[3 * o + a];
            d1[a] = x1 - c.L * rint(x1 * c.invL);
            d2[a] = x2 - c.L * rint(x2 * c.invL);
        }
        double r1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        double r2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
        double g1 = -kb * (r1 - r0) / r1, g2 = -kb * (r2 - r0) / r2;
        u += 0.5 * kb * (r1 - r0) * (r1 - r0) + 0.5 * kb * (r2 - r0) * (r2 - r0);
        double cth = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (r1 * r2);
        cth = fmin(1.0, fmax(-1.0, cth));
        double th = acos(cth);
        double sn = fmax(sqrt(1.0 - cth * cth), 1e-12);
        u += 0.5 * kth * (th - th0) * (th - th0);
        double dUdth = kth * (th - th0);
        double fo[3], fh1[3], fh2[3];
        for (int a = 0; a < 3; ++a) {
            double f1 = -dUdth * (-(d2[a] / (r1 * r2) - cth * d1[a] / (r1 * r1)) / sn);
            double f2 = -dUdth * (-(d1[a] / (r1 * r2) - cth * d2[a] / (r2 * r2)) / sn);
            fh1[a] = g1 * d1[a] + f1;
            fh2[a] = g2 * d2[a] + f2;
            fo[a] = -(g1 * d1[a] + g2 * d2[a]) - (f1 + f2);
        }
        for (int a = 0; a < 3; ++a) {
            Fb[3 * o + a] = fo[a];
            Fb[3 * (o + 1) + a] = fh1[a];
            Fb[3 * (o + 2) + a] = fh2[a];
        }
    }
    __shared__ double red[TPB / 32];
    u = warp_sum(u);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = u;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < TPB / 32; ++w) s += red[w];
        part[bx] = s;
    }
}

__global__ void __launch_bounds__(TPB) k_bonded(int nmol, const double* __restrict__ pos, RbeConsts c, double kb,
                                                double r0, double kth, double th0, double* __restrict__ Fb,
                                                double* __restrict__ part)
{
    bonded_body(blockIdx.x, gridDim.x, nmol, pos, c, kb, r0, kth, th0, Fb, part);
}

// Fixed-order block reduction of a strided column.
// Fixed-order block sum of one value per thread: a butterfly inside each warp
// (lane 0's result), then the warp results in warp order, read by every
// thread in the same order.  sh holds at least blockDim/32 doubles.
__device__ double block_reduce(double v, double* sh)
{
    v = warp_sum(v);
    __syncthreads();                      // earlier readers of sh are done
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    return r;
}

__device__ double block_sum_col(const double* __restrict__ src, int nrow, int stride, int col, double* sh)
{
    double s = 0.0;
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) s += src[(size_t)r * stride + col];
    return block_reduce(s, sh);
}

// totals: E[0..5], W[6..11], corr[12..14]
// The pair kernel's [grid][12] block partials are summed in RBE_FIN_CHUNKS
// fixed chunks of consecutive rows (one warp per chunk: lane l takes rows
// start + l, start + l + 32, ..., then a warp butterfly), so that the FP64
// additions spread over many SMs (GB300's FP64 pipe is narrow); one warp then
// sums the chunk results, the charge and k-term partials and the bond
// partials the same way (lane-strided rows, butterfly).  The batched form
// computes the same chunks with its block's warps and the same last warp sum,
// so both paths add in one fixed order.
constexpr int FIN_NV = RBE_NPART_RBL + RBE_NPART_Q + 7 + 1;
__device__ __forceinline__ void rbl_chunk_sum(int g, int R, const double* __restrict__ part_rbl,
                                              double* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int cs = (R + RBE_FIN_CHUNKS - 1) / RBE_FIN_CHUNKS;
    const int r0 = g * cs, r1 = min(R, r0 + cs);
    double v[RBE_NPART_RBL];
#pragma unroll
    for (int q = 0; q < RBE_NPART_RBL; ++q) v[q] = 0.0;
    for (int r = r0 + lane; r < r1; r += 32) {
        const double* row = part_rbl + (size_t)r * RBE_NPART_RBL;
#pragma unroll
        for (int q = 0; q < RBE_NPART_RBL; ++q) v[q] += row[q];
    }
#pragma unroll
    for (int q = 0; q < RBE_NPART_RBL; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0)
        for (int q = 0; q < RBE_NPART_RBL; ++q) out[g * RBE_NPART_RBL + q] = v[q];
}

// one warp: the totals from the chunk sums and the other partials
__device__ __forceinline__ void finalize_warp(int n, const RbeConsts& c, const double* __restrict__ chunks,
                                              const double* __restrict__ part_q, int grid_q,
                                              const double* __restrict__ kterms, const double* __restrict__ part_bond,
                                              int grid_bond, double* __restrict__ totals, int* __restrict__ status)
{
    const int lane = threadIdx.x & 31;
    double v[FIN_NV];
#pragma unroll
    for (int q = 0; q < FIN_NV; ++q) v[q] = 0.0;
    // (the loops are unrolled so that several rows' loads are in flight)
#pragma unroll
    for (int g = lane; g < RBE_FIN_CHUNKS; g += 32) {
#pragma unroll
        for (int q = 0; q < RBE_NPART_RBL; ++q) v[q] += chunks[g * RBE_NPART_RBL + q];
    }
#pragma unroll 8
    for (int r = lane; r < grid_q; r += 32) {
#pragma unroll
        for (int q = 0; q < RBE_NPART_Q; ++q) v[RBE_NPART_RBL + q] += part_q[(size_t)r * RBE_NPART_Q + q];
    }
#pragma unroll 4
    for (int r = lane; r < c.P; r += 32) {
#pragma unroll
        for (int q = 0; q < 7; ++q) v[RBE_NPART_RBL + RBE_NPART_Q + q] += kterms[(size_t)r * 7 + q];
    }
    for (int r = lane; r < grid_bond; r += 32) v[FIN_NV - 1] += part_bond[r];
#pragma unroll
    for (int q = 0; q < FIN_NV; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0) {
        const double* r = v;
        const double* qs = v + RBE_NPART_RBL;
        const double* kt = qs + RBE_NPART_Q;
        const double eb = v[FIN_NV - 1];
        totals[0] = 0.5 * r[0];
        totals[1] = kt[0];
        totals[2] = -c.k_e * sqrt(c.alpha / 3.14159265358979323846) * qs[0];
        totals[3] = 0.5 * r[1];
        totals[4] = 0.5 * r[2];
        totals[5] = eb;
        for (int a = 0; a < 6; ++a) totals[6 + a] = -0.5 * r[3 + a] + kt[1 + a];
        for (int a = 0; a < 3; ++a) totals[12 + a] = r[9 + a] / (double)n;
        if (fabs(qs[1]) > 1e-10 * qs[2]) latch_status(status, RBE_ST_NONNEUTRAL);
        bool fin = true;
        for (int a = 0; a < 15; ++a) fin = fin && isfinite(totals[a]);
        if (!fin) latch_status(status, RBE_ST_NONFINITE);
    }
}

// RBE_FIN_CHUNKS blocks of one warp
__global__ void __launch_bounds__(32) k_fin_chunks(int grid_rbl, const double* __restrict__ part_rbl,
                                                   double* __restrict__ chunks)
{
    rbl_chunk_sum(blockIdx.x, grid_rbl, part_rbl, chunks);
}

// one warp
__global__ void __launch_bounds__(32) k_finalize(int n, RbeConsts c, const double* __restrict__ chunks,
                                                 const double* __restrict__ part_q, int grid_q,
                                                 const double* __restrict__ kterms,
                                                 const double* __restrict__ part_bond, int grid_bond,
                                                 double* __restrict__ totals, int* __restrict__ status)
{
    finalize_warp(n, c, chunks, part_q, grid_q, kterms, part_bond, grid_bond, totals, status);
}

template <bool MIXED>
__device__ __forceinline__ void kforce_body(int bx, int n, const RbeConsts& c, const uint4* __restrict__ s4,
                                            const double4_32a* __restrict__ p4, const int* __restrict__ perm,
                                            const int4* __restrict__ km, const double4_32a* __restrict__ kv,
                                            const double2* __restrict__ cis,
                                            const double2* __restrict__ rho, const double* __restrict__ F_real,
                                            const double* __restrict__ totals, const double* __restrict__ F_bond,
                                            int n_bonded_atoms, double* __restrict__ F)
{
    constexpr int KT = 256;
    __shared__ double4_32a sk_d[MIXED ? 1 : KT];      // kx, ky, kz, unused
    __shared__ double2 sab_d[MIXED ? 1 : KT];     // (c Im rho, c Re rho)
    __shared__ int4 sm[KT];
    __shared__ float4 sk_f[MIXED ? KT : 1];       // kx, ky, kz, c Im rho (mixed: sm[k].w holds c Re rho)
    const int i = bx * TPB + threadIdx.x;
    const bool act = i < n;
    uint4 si = make_uint4(0, 0, 0, 0);
    double4_32a pi = make_double4_32a(0, 0, 0, 0);
    uint64_t sxi = 0, syi = 0, szi = 0;         // FP64: 64-bit codes of the position
    if (act) {
        si = s4[i];
        if (!MIXED) {
            pi = p4[i];
            sxi = code64_of(pi.x, c.invL);
            syi = code64_of(pi.y, c.invL);
            szi = code64_of(pi.z, c.invL);
        }
    }
    double f[3] = {0.0, 0.0, 0.0};
    float fm[3] = {0.f, 0.f, 0.f};        // mixed: the Fourier sums in FP32
    for (int l0 = 0; l0 < c.P; l0 += KT) {
        const int cnt = min(KT, c.P - l0);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += TPB) {
            double4_32a k4 = kv[l0 + k];
            double2 r = rho[l0 + k];
            if (MIXED) {
                const int4 mk = km[l0 + k];
                sm[k] = make_int4(mk.x, mk.y, mk.z, __float_as_int((float)(k4.w * r.x)));
                sk_f[k] = make_float4((float)k4.x, (float)k4.y, (float)k4.z, (float)(k4.w * r.y));
            } else {
                sm[k] = km[l0 + k];
                sk_d[k] = k4;
                sab_d[k] = make_double2(k4.w * r.y, k4.w * r.x);
            }
        }
        __syncthreads();
        if (act) {
            if (MIXED) {
                float g[3] = {0.f, 0.f, 0.f};
                for (int k = 0; k < cnt; ++k) {
                    int4 m = sm[k];
                    uint32_t ph = (uint32_t)m.x * si.x + (uint32_t)m.y * si.y + (uint32_t)m.z * si.z;
                    float ang = (float)(int)ph * 1.4629180792671596e-09f;
                    float sn, cs;
                    __sincosf(ang, &sn, &cs);
                    float4 kk = sk_f[k];
                    // Im(e^{-i th} rho) c = cos(th) c Im rho - sin(th) c Re rho
                    float h = cs * kk.w - sn * __int_as_float(m.w);
                    g[0] += h * kk.x; g[1] += h * kk.y; g[2] += h * kk.z;
                }
                for (int a = 0; a < 3; ++a) fm[a] += g[a];
            } else {
                for (int k = 0; k < cnt; ++k) {
                    const int4 m = sm[k];
                    const double4_32a kk = sk_d[k];
                    const uint64_t ph = (uint64_t)(long long)m.x * sxi + (uint64_t)(long long)m.y * syi +
                                        (uint64_t)(long long)m.z * szi;
                    double sn, cs;
                    cis_fp64_64(ph, cis, cs, sn);
                    const double2 ab = sab_d[k];
                    const double h = cs * ab.x - sn * ab.y;
                    f[0] += h * kk.x; f[1] += h * kk.y; f[2] += h * kk.z;
                }
            }
        }
    }
    if (!act) return;
    if (MIXED) {
        // the mixed forces are combined in FP32 (F_real, the Fourier sums and
        // the charge are FP32 already) and widened once: the FP64 pipe of
        // this part is narrow, and the result keeps the mixed path's bar
        const float qf = __uint_as_float(si.w);
        const int gi = perm[i];
        const float* Fr = reinterpret_cast<const float*>(F_real) + 3 * (size_t)i;
        for (int a = 0; a < 3; ++a) {
            double v = (double)(Fr[a] - (float)totals[12 + a] - qf * fm[a]);
            if (gi < n_bonded_atoms) v += F_bond[3 * (size_t)gi + a];
            F[3 * (size_t)gi + a] = v;
        }
        return;
    }
    const double qi = pi.w;
    const int gi = perm[i];
    for (int a = 0; a < 3; ++a) {
        double fr = MIXED ? (double)reinterpret_cast<const float*>(F_real)[3 * (size_t)i + a] : F_real[3 * (size_t)i + a];
        double v = fr - totals[12 + a] - qi * f[a];
        if (gi < n_bonded_atoms) v += F_bond[3 * (size_t)gi + a];
        F[3 * (size_t)gi + a] = v;
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(TPB) k_kforce(int n, RbeConsts c, const uint4* __restrict__ s4,
                                                const double4_32a* __restrict__ p4, const int* __restrict__ perm,
                                                const int4* __restrict__ km, const double4_32a* __restrict__ kv,
                                                const double2* __restrict__ cis, const double2* __restrict__ rho, const double* __restrict__ F_real,
                                                const double* __restrict__ totals, const double* __restrict__ F_bond,
                                                int n_bonded_atoms, double* __restrict__ F)
{
    kforce_body<MIXED>(blockIdx.x, n, c, s4, p4, perm, km, kv, cis, rho, F_real, totals, F_bond, n_bonded_atoms, F);
}

// Half kick v += (dt/2) accel (F + F^L) / m (F^L the Langevin force, or none)
// and, with drift, x += dt v.
__device__ __forceinline__ void vv_body(int bx, int n, double* __restrict__ pos, double* __restrict__ vel,
                                        const double* __restrict__ mass, const double* __restrict__ F,
                                        const double* __restrict__ FL, double hdta, double dt, int drift)
{
    int i = bx * TPB + threadIdx.x;
    if (i >= n) return;
    double m = mass[i];
    for (int a = 0; a < 3; ++a) {
        const double f = FL ? __dadd_rn(F[3 * i + a], FL[3 * i + a]) : F[3 * i + a];
        double v = __dadd_rn(vel[3 * i + a], __ddiv_rn(__dmul_rn(hdta, f), m));
        vel[3 * i + a] = v;
        if (drift) pos[3 * i + a] = __dadd_rn(pos[3 * i + a], __dmul_rn(dt, v));
    }
}

// rbe_step's kick: once an error is latched (by the force evaluation it
// would use, or earlier) it leaves positions and velocities as they are and
// records its code (2k first half kick and drift of step k, 2k + 1 second
// half kick) if it is the first to stop
__global__ void __launch_bounds__(TPB) k_vv(int n, double* __restrict__ pos, double* __restrict__ vel,
                                            const double* __restrict__ mass, const double* __restrict__ F,
                                            const double* __restrict__ FL, double hdta, double dt, int drift,
                                            int* __restrict__ status, int code)
{
    if (*(volatile int*)status != 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(status + RBE_STW_HALT, -1, code);
        return;
    }
    vv_body(blockIdx.x, n, pos, vel, mass, F, FL, hdta, dt, drift);
}

// Langevin thermostat (Sec. 3.1 runs its electrolytes with one, relaxation
// time tau, inside velocity Verlet): at the force evaluation of step s,
//   F^L_i = -(m_i / c1) v_i + sqrt(m_i c2) (u - 1/2),  c1 = accel tau,
//   c2 = 24 kT / (c1 dt),
// a uniform random force of variance 2 m kT / (accel tau dt) per component
// (the Euler-Maruyama impulse), u = (w >> 11) 2^-53 from word a of the Philox
// block at counter (i, 0, s, 3), i the caller's atom index.
__device__ __forceinline__ void langevin_body(int bx, int n, const double* __restrict__ vel,
                                              const double* __restrict__ mass, uint64_t seed, uint64_t s, double c1,
                                              double c2, double* __restrict__ FL)
{
    const int i = bx * TPB + threadIdx.x;
    if (i >= n) return;
    uint64_t w[4];
    philox4x64_10((uint64_t)i, 0ull, s, 3ull, seed, 0ull, w);
    const double m = mass[i];
    const double amp = __dsqrt_rn(__dmul_rn(m, c2));
    const double fr = __ddiv_rn(m, c1);
    for (int a = 0; a < 3; ++a) {
        const double u = __dmul_rn((double)(w[a] >> 11), 1.1102230246251565e-16);
        FL[3 * i + a] = __dadd_rn(__dmul_rn(-fr, vel[3 * i + a]), __dmul_rn(amp, __dsub_rn(u, 0.5)));
    }
}

__global__ void __launch_bounds__(TPB) k_langevin(int n, const double* __restrict__ vel,
                                                  const double* __restrict__ mass, uint64_t seed, uint64_t s,
                                                  double c1, double c2, double* __restrict__ FL)
{
    langevin_body(blockIdx.x, n, vel, mass, seed, s, c1, c2, FL);
}

__device__ __forceinline__ void ke_body(int bx, int nbx, int n, const double* __restrict__ vel,
                                        const double* __restrict__ mass, double* __restrict__ part)
{
    double s = 0.0;
    for (int i = bx * TPB + threadIdx.x; i < n; i += nbx * TPB)
        for (int a = 0; a < 3; ++a) s += 0.5 * mass[i] * vel[3 * i + a] * vel[3 * i + a];
    __shared__ double red[TPB / 32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < TPB / 32; ++w) t += red[w];
        part[bx] = t;
    }
}

__global__ void __launch_bounds__(TPB) k_ke(int n, const double* __restrict__ vel, const double* __restrict__ mass,
                                            double* __restrict__ part)
{
    ke_body(blockIdx.x, gridDim.x, n, vel, mass, part);
}

__device__ __forceinline__ void trace_body(const double* __restrict__ part, int nblk, const double* __restrict__ totals,
                                           double accel, double* __restrict__ out)
{
    __shared__ double sh[TPB];
    double ke = block_sum_col(part, nblk, 1, 0, sh);
    if (threadIdx.x == 0) {
        out[0] = totals[0] + totals[1] + totals[2] + totals[3] + totals[4] + totals[5];
        out[1] = ke / accel;
    }
}

__global__ void __launch_bounds__(TPB) k_trace(const double* __restrict__ part, int nblk, const double* __restrict__ totals,
                                               double accel, double* __restrict__ out)
{
    trace_body(part, nblk, totals, accel, out);
}

// ---- batched forms: one launch over all replicas of a plan -----------------
// Per-replica grids: BK_KS = ceil(P / TPB) (sampling), BK_RS = ceil(P / 8)
// (rho sum, a warp per k), BK_RHO = grid_rho, BK_BOND = grid_bond (0 without
// bonds), BK_ATOMS = ceil(n / TPB), BK_Q = grid_q, BK_REP = 1.

__global__ void k_ctl_b(BatchCtl* ctl, int op, unsigned long long step0, double* trace, int nsteps)
{
    if (op == 0) {          // set: the next batched step uses step0
        ctl->step = step0;
        ctl->step0 = step0;
        ctl->trace = trace;
        ctl->nsteps = nsteps;
    } else if (op == 1) {   // advance by one MD step
        ctl->step += 1;
    }
    ctl->rbl_next = 0;      // every op empties the pair kernel's work queue
}

__global__ void __launch_bounds__(TPB) k_sample_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep,
                                                  const BatchCtl* __restrict__ ctl)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    sample_body(bx, nbx, d.c, ctl->step, d.kT, d.kpool, d.km, d.kv, d.status);
}

template <bool MIXED>
__global__ void k_rho_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    rho_body<MIXED>(bx, d.n, d.rho_chunk, d.c, d.s4, d.p4, d.km, d.kv, d.cis, d.rho_part);
}

__global__ void __launch_bounds__(TPB) k_rho_sum_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep)  // BK_RS
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    rho_sum_body(bx, d.grid_rho, d.c, d.rho_part, d.kv, d.rho, d.totals + 32);
}

__global__ void __launch_bounds__(TPB) k_bonded_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    bonded_body(bx, nbx, d.nmol, d.pos, d.c, d.kb, d.r0, d.kth, d.th0, d.F_bond, d.part_bond);
}

__global__ void __launch_bounds__(FIN_TPB) k_finalize_b(const RepDev* __restrict__ R)
{
    __shared__ double chunks[RBE_FIN_CHUNKS * RBE_NPART_RBL];
    const RepDev& d = R[blockIdx.x];
    for (int g = threadIdx.x >> 5; g < RBE_FIN_CHUNKS; g += FIN_TPB / 32) rbl_chunk_sum(g, d.grid_rbl, d.part_rbl, chunks);
    __syncthreads();
    if (threadIdx.x < 32)
        finalize_warp(d.n, d.c, chunks, d.part_q, d.grid_q, d.totals + 32, d.part_bond, d.grid_bond, d.totals,
                      d.status);
}

template <bool MIXED>
__global__ void __launch_bounds__(TPB) k_kforce_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    kforce_body<MIXED>(bx, d.n, d.c, d.s4, d.p4, d.perm, d.km, d.kv, d.cis, d.rho, d.F_real, d.totals, d.F_bond,
                       d.n_bonded_atoms, d.F);
}

__global__ void __launch_bounds__(TPB) k_vv_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep,
                                              int drift)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    vv_body(bx, d.n, d.pos, d.vel, d.mass, d.F, d.FL, 0.5 * d.dt * d.accel, d.dt, drift);
}

// mask (may be null: every replica): replicas whose force is (re)computed
__global__ void __launch_bounds__(TPB) k_langevin_b(const RepDev* __restrict__ R, const int* __restrict__ off,
                                                    int nrep, const BatchCtl* __restrict__ ctl,
                                                    const int* __restrict__ mask)
{
    int bx, nbx;
    const int r = rep_of_block(off, nrep, blockIdx.x, bx, nbx);
    const RepDev& d = R[r];
    if (!d.FL || (mask && !mask[r])) return;
    langevin_body(bx, d.n, d.vel, d.mass, d.c.seed, ctl->step, d.lang_c1, d.lang_c2, d.FL);
}

__global__ void __launch_bounds__(TPB) k_ke_b(const RepDev* __restrict__ R, const int* __restrict__ off, int nrep)
{
    int bx, nbx;
    const RepDev& d = R[rep_of_block(off, nrep, blockIdx.x, bx, nbx)];
    ke_body(bx, nbx, d.n, d.vel, d.mass, d.ke_part);
}

// Trace entry k = step - step0 - 1 of replica r: [potential, kinetic / accel].
__global__ void __launch_bounds__(TPB) k_trace_b(const RepDev* __restrict__ R, const BatchCtl* __restrict__ ctl)
{
    const RepDev& d = R[blockIdx.x];
    const long long k = (long long)(ctl->step - ctl->step0) - 1;
    if (!ctl->trace || k < 0 || k >= ctl->nsteps) return;
    trace_body(d.ke_part, d.grid_q, d.totals, d.accel,
               ctl->trace + ((size_t)blockIdx.x * ctl->nsteps + (size_t)k) * 2);
}

}  // namespace

void launch_ksample(rbe_ctx* ctx, uint64_t step, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_KSAMPLE, st);
    int g = (ctx->c.P + TPB - 1) / TPB;
    k_sample<<<g, TPB, 0, st>>>(ctx->c, step, ctx->kT, ctx->kpool_buf, ctx->km, ctx->kv, ctx->status);
    prof_end(ctx, RBE_K_KSAMPLE, st);
}

void launch_kpool_build(rbe_ctx* ctx, const double* w, const double* q, const uint64_t* Tq, int M, cudaStream_t st)
{
    k_kpool_build<<<1, 32, 0, st>>>(ctx->c.seed, M, ctx->c.kpool, ctx->kpool_burn, w, q, Tq, ctx->kpool_buf,
                                    ctx->status);
}

void launch_cis_table(double2* tab, cudaStream_t st)
{
    k_cis_table<<<256, 256, 0, st>>>(tab);
}

void launch_rho(rbe_ctx* ctx, int n, cudaStream_t st)
{
    int P = ctx->c.P;
    int threads = ((P < 1024 ? P : 1024) + 31) / 32 * 32;
    int chunk = (n + ctx->grid_rho - 1) / ctx->grid_rho;
    prof_begin(ctx, RBE_K_RHO, st);
    if (ctx->precision == RBE_MIXED)
        k_rho<true><<<ctx->grid_rho, threads, 0, st>>>(n, chunk, ctx->c, ctx->s4, ctx->p4, ctx->km, ctx->kv, ctx->cis,
                                                         ctx->rho_part);
    else
        k_rho<false><<<ctx->grid_rho, threads, 0, st>>>(n, chunk, ctx->c, ctx->s4, ctx->p4, ctx->km, ctx->kv, ctx->cis,
                                                          ctx->rho_part);
    prof_end(ctx, RBE_K_RHO, st);
    prof_begin(ctx, RBE_K_RHOSUM, st);
    double* kterms = ctx->totals + 32;
    k_rho_sum<<<(P + TPB / 32 - 1) / (TPB / 32), TPB, 0, st>>>(ctx->grid_rho, ctx->c, ctx->rho_part, ctx->kv, ctx->rho,
                                                                kterms);
    prof_end(ctx, RBE_K_RHOSUM, st);
}

void launch_bonded(rbe_ctx* ctx, int n, const double* pos, cudaStream_t st)
{
    (void)n;
    prof_begin(ctx, RBE_K_BONDED, st);
    k_bonded<<<ctx->grid_bond, TPB, 0, st>>>(ctx->n_wmol, pos, ctx->c, ctx->kb, ctx->r0, ctx->kth, ctx->th0, ctx->F_bond,
                                             ctx->part_bond);
    prof_end(ctx, RBE_K_BONDED, st);
}

void launch_finalize(rbe_ctx* ctx, int n, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_FINAL, st);
    k_fin_chunks<<<RBE_FIN_CHUNKS, 32, 0, st>>>(ctx->grid_rbl, ctx->part_rbl, ctx->fin_part);
    k_finalize<<<1, 32, 0, st>>>(n, ctx->c, ctx->fin_part, ctx->part_q, ctx->grid_q, ctx->totals + 32,
                                  ctx->part_bond, ctx->n_wmol > 0 ? ctx->grid_bond : 0, ctx->totals, ctx->status);
    prof_end(ctx, RBE_K_FINAL, st);
}

void launch_kforce(rbe_ctx* ctx, int n, double* F, cudaStream_t st)
{
    int g = (n + TPB - 1) / TPB;
    int nb = ctx->n_wmol > 0 ? 3 * ctx->n_wmol : 0;
    prof_begin(ctx, RBE_K_KFORCE, st);
    if (ctx->precision == RBE_MIXED)
        k_kforce<true><<<g, TPB, 0, st>>>(n, ctx->c, ctx->s4, ctx->p4, ctx->perm, ctx->km, ctx->kv, ctx->cis, ctx->rho,
                                          ctx->F_real, ctx->totals, ctx->F_bond, nb, F);
    else
        k_kforce<false><<<g, TPB, 0, st>>>(n, ctx->c, ctx->s4, ctx->p4, ctx->perm, ctx->km, ctx->kv, ctx->cis, ctx->rho,
                                           ctx->F_real, ctx->totals, ctx->F_bond, nb, F);
    prof_end(ctx, RBE_K_KFORCE, st);
}

void launch_vv_kick_drift(rbe_ctx* ctx, int n, double* pos, double* vel, const double* mass, const double* F,
                          const double* FL, double dt, double accel, int drift, int code, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_VV, st);
    k_vv<<<(n + TPB - 1) / TPB, TPB, 0, st>>>(n, pos, vel, mass, F, FL, 0.5 * dt * accel, dt, drift, ctx->status,
                                              code);
    prof_end(ctx, RBE_K_VV, st);
}

void launch_langevin(rbe_ctx* ctx, int n, const double* vel, const double* mass, uint64_t s, double dt, double accel,
                     cudaStream_t st)
{
    const double c1 = accel * ctx->lang_tau;
    const double c2 = 24.0 * ctx->lang_kT / (c1 * dt);
    prof_begin(ctx, RBE_K_VV, st);
    k_langevin<<<(n + TPB - 1) / TPB, TPB, 0, st>>>(n, vel, mass, ctx->c.seed, s, c1, c2, ctx->F_lang);
    prof_end(ctx, RBE_K_VV, st);
}

void launch_ke_trace(rbe_ctx* ctx, int n, const double* vel, const double* mass, double accel, double* trace_slot,
                     cudaStream_t st)
{
    prof_begin(ctx, RBE_K_MISC, st);
    k_ke<<<ctx->grid_q, TPB, 0, st>>>(n, vel, mass, ctx->ke_part);
    prof_end(ctx, RBE_K_MISC, st);
    prof_begin(ctx, RBE_K_MISC, st);
    k_trace<<<1, TPB, 0, st>>>(ctx->ke_part, ctx->grid_q, ctx->totals, accel, trace_slot);
    prof_end(ctx, RBE_K_MISC, st);
}

void launch_ctl_batch(const BatchPlan& bp, int op, unsigned long long step0, double* trace, int nsteps,
                      cudaStream_t st)
{
    k_ctl_b<<<1, 1, 0, st>>>(bp.ctl, op, step0, trace, nsteps);
}

void launch_kspace_pre_batch(const BatchPlan& bp, cudaStream_t st)
{
    const int nr = bp.nrep;
    k_sample_b<<<bp.total[BK_KS], TPB, 0, st>>>(bp.rep, bp.off[BK_KS], nr, bp.ctl);
    if (bp.precision == RBE_MIXED)
        k_rho_b<true><<<bp.total[BK_RHO], bp.rho_threads, 0, st>>>(bp.rep, bp.off[BK_RHO], nr);
    else
        k_rho_b<false><<<bp.total[BK_RHO], bp.rho_threads, 0, st>>>(bp.rep, bp.off[BK_RHO], nr);
    k_rho_sum_b<<<bp.total[BK_RS], TPB, 0, st>>>(bp.rep, bp.off[BK_RS], nr);
    if (bp.total[BK_BOND] > 0) k_bonded_b<<<bp.total[BK_BOND], TPB, 0, st>>>(bp.rep, bp.off[BK_BOND], nr);
}

void launch_kspace_post_batch(const BatchPlan& bp, cudaStream_t st)
{
    const int nr = bp.nrep;
    k_finalize_b<<<nr, FIN_TPB, 0, st>>>(bp.rep);
    if (bp.precision == RBE_MIXED)
        k_kforce_b<true><<<bp.total[BK_ATOMS], TPB, 0, st>>>(bp.rep, bp.off[BK_ATOMS], nr);
    else
        k_kforce_b<false><<<bp.total[BK_ATOMS], TPB, 0, st>>>(bp.rep, bp.off[BK_ATOMS], nr);
}

void launch_vv_batch(const BatchPlan& bp, int drift, cudaStream_t st)
{
    k_vv_b<<<bp.total[BK_ATOMS], TPB, 0, st>>>(bp.rep, bp.off[BK_ATOMS], bp.nrep, drift);
}

void launch_langevin_batch(const BatchPlan& bp, const int* mask, cudaStream_t st)
{
    k_langevin_b<<<bp.total[BK_ATOMS], TPB, 0, st>>>(bp.rep, bp.off[BK_ATOMS], bp.nrep, bp.ctl, mask);
}

void launch_ke_trace_batch(const BatchPlan& bp, cudaStream_t st)
{
    k_ke_b<<<bp.total[BK_Q], TPB, 0, st>>>(bp.rep, bp.off[BK_Q], bp.nrep);
    k_trace_b<<<bp.nrep, TPB, 0, st>>>(bp.rep, bp.ctl);
}

// ---------------------------------------------------------------------------
// Adjoint of the force step (gradients with the draws frozen)
// ---------------------------------------------------------------------------
namespace {

// Upstream force gradient into sorted order, with block sums for its mean.
__global__ void __launch_bounds__(TPB) k_gather_v(int n, const int* __restrict__ perm, const double* __restrict__ gF,
                                                  double* __restrict__ vs, double* __restrict__ part_v)
{
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = blockIdx.x * TPB + threadIdx.x; k < n; k += gridDim.x * TPB) {
        const int i = perm[k];
        for (int a = 0; a < 3; ++a) {
            const double v = gF ? gF[3 * (size_t)i + a] : 0.0;
            vs[3 * (size_t)k + a] = v;
            s[a] += v;
        }
    }
    __shared__ double red[3][TPB / 32];
    for (int a = 0; a < 3; ++a) s[a] = warp_sum(s[a]);
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) red[a][threadIdx.x >> 5] = s[a];
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < TPB / 32; ++w) t += red[threadIdx.x][w];
        part_v[blockIdx.x * 3 + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(TPB) k_vbar(int n, int nblk, const double* __restrict__ part_v,
                                              double* __restrict__ totals)
{
    __shared__ double sh[TPB];
    for (int a = 0; a < 3; ++a) {
        const double s = block_sum_col(part_v, nblk, 3, a, sh);
        if (threadIdx.x == 0) totals[16 + a] = s / (double)n;
    }
}

// tau_l = sum_i q_i (v_i . k_l) exp(i k_l . r_i): block partials, as k_rho.
template <bool MIXED>
__global__ void k_tau(int n, int chunk, RbeConsts c, const uint4* __restrict__ s4, const double4_32a* __restrict__ p4,
                      const double* __restrict__ vs, const int4* __restrict__ km, const double4_32a* __restrict__ kv,
                      const double2* __restrict__ cis, double2* __restrict__ part)
{
    __shared__ double4_32a tile_d[TILE];
    __shared__ double tile_v[TILE][3];
    __shared__ double tile_r[MIXED ? 1 : TILE][3];    // FP64: residuals of the fixed-point codes
    __shared__ uint4 tile_u[TILE];
    const int b0 = blockIdx.x * chunk;
    const int b1 = min(n, b0 + chunk);
    for (int l0 = 0; l0 < c.P; l0 += blockDim.x) {
        const int l = l0 + threadIdx.x;
        const bool act = l < c.P;
        const int4 m = act ? km[l] : make_int4(0, 0, 0, 0);
        const double4_32a k = act ? kv[l] : make_double4_32a(0, 0, 0, 0);
        double re = 0.0, im = 0.0;
        for (int t0 = b0; t0 < b1; t0 += TILE) {
            const int cnt = min(TILE, b1 - t0);
            __syncthreads();
            for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
                const double4_32a pe = p4[t0 + e];
                const uint4 se = s4[t0 + e];
                tile_d[e] = pe;
                tile_u[e] = se;
                if (!MIXED) {
                    const double Lq = c.L * 2.3283064365386963e-10;
                    tile_r[e][0] = fixed_residual(pe.x, se.x, Lq);
                    tile_r[e][1] = fixed_residual(pe.y, se.y, Lq);
                    tile_r[e][2] = fixed_residual(pe.z, se.z, Lq);
                }
                for (int a = 0; a < 3; ++a) tile_v[e][a] = vs[3 * (size_t)(t0 + e) + a];
            }
            __syncthreads();
            if (act) {
                for (int e = 0; e < cnt; ++e) {
                    const double4_32a p = tile_d[e];
                    const double wv = p.w * (k.x * tile_v[e][0] + k.y * tile_v[e][1] + k.z * tile_v[e][2]);
                    double sn, cs;
                    if (MIXED) {
                        const uint4 s = tile_u[e];
                        const uint32_t ph = (uint32_t)m.x * s.x + (uint32_t)m.y * s.y + (uint32_t)m.z * s.z;
                        float fs, fc;
                        __sincosf((float)(int)ph * 1.4629180792671596e-09f, &fs, &fc);
                        sn = fs; cs = fc;
                    } else {
                        const uint4 s = tile_u[e];
                        const uint32_t ph = (uint32_t)m.x * s.x + (uint32_t)m.y * s.y + (uint32_t)m.z * s.z;
                        cis_fp64(ph, fma(k.x, tile_r[e][0], fma(k.y, tile_r[e][1], k.z * tile_r[e][2])), cis, cs, sn);
                    }
                    re += wv * cs;
                    im += wv * sn;
                }
            }
        }
        if (act) part[(size_t)blockIdx.x * c.P + l] = make_double2(re, im);
    }
}

__global__ void __launch_bounds__(TPB) k_tau_sum(int nblk, int P, const double2* __restrict__ part,
                                                 double2* __restrict__ tau)
{
    const int l = blockIdx.x * TPB + threadIdx.x;
    if (l >= P) return;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nblk; ++b) {
        const double2 v = part[(size_t)b * P + l];
        re += v.x;
        im += v.y;
    }
    tau[l] = make_double2(re, im);
}

// Per atom: Fourier and self parts, plus the pair parts, into caller order.
//   dE_k/dq_i = sum_l c_l Re(conj(rho_l) e^{i th}),  dE_self/dq_i = -2 k_e sqrt(a/pi) q_i
//   dL/dq_i  -= sum_l c_l [(v_i . k_l) Im(e^{-i th} rho_l) + Im(e^{i th} conj(tau_l))]
template <bool MIXED>
__global__ void __launch_bounds__(TPB) k_kadj(int n, RbeConsts c, const uint4* __restrict__ s4,
                                              const double4_32a* __restrict__ p4, const int* __restrict__ perm,
                                              const int4* __restrict__ km, const double4_32a* __restrict__ kv,
                                              const double2* __restrict__ cis,
                                              const double2* __restrict__ rho, const double2* __restrict__ tau,
                                              const double* __restrict__ vs, const double* __restrict__ gq_own,
                                              const double* __restrict__ gq_tr, double* __restrict__ dEdq,
                                              double* __restrict__ dLdq)
{
    constexpr int KT = 128;
    __shared__ double4_32a sk[KT];
    __shared__ int4 sm[KT];
    __shared__ double4_32a srt[KT];   // rho re, rho im, tau re, tau im
    const int i = blockIdx.x * TPB + threadIdx.x;
    const bool act = i < n;
    const double4_32a pi = act ? p4[i] : make_double4_32a(0, 0, 0, 0);
    const uint4 si = act ? s4[i] : make_uint4(0, 0, 0, 0);
    const double Lq = c.L * 2.3283064365386963e-10;
    const double rxi = MIXED ? 0.0 : fixed_residual(pi.x, si.x, Lq);
    const double ryi = MIXED ? 0.0 : fixed_residual(pi.y, si.y, Lq);
    const double rzi = MIXED ? 0.0 : fixed_residual(pi.z, si.z, Lq);
    const double vx = act ? vs[3 * (size_t)i] : 0.0, vy = act ? vs[3 * (size_t)i + 1] : 0.0;
    const double vz = act ? vs[3 * (size_t)i + 2] : 0.0;
    double gE = 0.0, gL = 0.0;
    for (int l0 = 0; l0 < c.P; l0 += KT) {
        const int cnt = min(KT, c.P - l0);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += TPB) {
            sk[k] = kv[l0 + k];
            sm[k] = km[l0 + k];
            const double2 r = rho[l0 + k], t = tau[l0 + k];
            srt[k] = make_double4_32a(r.x, r.y, t.x, t.y);
        }
        __syncthreads();
        if (act) {
            for (int k = 0; k < cnt; ++k) {
                const double4_32a kk = sk[k];
                double sn, cs;
                if (MIXED) {
                    const int4 m = sm[k];
                    const uint32_t ph = (uint32_t)m.x * si.x + (uint32_t)m.y * si.y + (uint32_t)m.z * si.z;
                    float fs, fc;
                    __sincosf((float)(int)ph * 1.4629180792671596e-09f, &fs, &fc);
                    sn = fs; cs = fc;
                } else {
                    const int4 m = sm[k];
                    const uint32_t ph = (uint32_t)m.x * si.x + (uint32_t)m.y * si.y + (uint32_t)m.z * si.z;
                    cis_fp64(ph, fma(kk.x, rxi, fma(kk.y, ryi, kk.z * rzi)), cis, cs, sn);
                }
                const double4_32a rt = srt[k];
                gE += kk.w * (rt.x * cs + rt.y * sn);
                const double vk = vx * kk.x + vy * kk.y + vz * kk.z;
                const double im1 = cs * rt.y - sn * rt.x;
                const double im2 = sn * rt.z - cs * rt.w;
                gL -= kk.w * (vk * im1 + im2);
            }
        }
    }
    if (!act) return;
    const int gi = perm[i];
    const double self = -2.0 * c.k_e * sqrt(c.alpha / 3.14159265358979323846) * pi.w;
    if (dEdq) dEdq[gi] = gE + self + gq_own[2 * (size_t)i] + gq_tr[2 * (size_t)i];
    if (dLdq) dLdq[gi] = gL + gq_own[2 * (size_t)i + 1] + gq_tr[2 * (size_t)i + 1];
}

}  // namespace

void launch_adj_prep(rbe_ctx* ctx, int n, const double* gF, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_MISC, st);
    k_gather_v<<<ctx->grid_q, TPB, 0, st>>>(n, ctx->perm, gF, ctx->vs, ctx->part_v);
    prof_end(ctx, RBE_K_MISC, st);
    prof_begin(ctx, RBE_K_MISC, st);
    k_vbar<<<1, TPB, 0, st>>>(n, ctx->grid_q, ctx->part_v, ctx->totals);
    prof_end(ctx, RBE_K_MISC, st);
    const int P = ctx->c.P;
    const int threads = ((P < 1024 ? P : 1024) + 31) / 32 * 32;
    const int chunk = (n + ctx->grid_rho - 1) / ctx->grid_rho;
    prof_begin(ctx, RBE_K_RHO, st);
    if (ctx->precision == RBE_MIXED)
        k_tau<true><<<ctx->grid_rho, threads, 0, st>>>(n, chunk, ctx->c, ctx->s4, ctx->p4, ctx->vs, ctx->km, ctx->kv,
                                                       ctx->cis, ctx->tau_part);
    else
        k_tau<false><<<ctx->grid_rho, threads, 0, st>>>(n, chunk, ctx->c, ctx->s4, ctx->p4, ctx->vs, ctx->km, ctx->kv,
                                                        ctx->cis, ctx->tau_part);
    prof_end(ctx, RBE_K_RHO, st);
    prof_begin(ctx, RBE_K_RHOSUM, st);
    k_tau_sum<<<(P + TPB - 1) / TPB, TPB, 0, st>>>(ctx->grid_rho, P, ctx->tau_part, ctx->tau);
    prof_end(ctx, RBE_K_RHOSUM, st);
}

void launch_adj_final(rbe_ctx* ctx, int n, double* dEdq, double* dLdq, cudaStream_t st)
{
    prof_begin(ctx, RBE_K_KFORCE, st);
    if (ctx->precision == RBE_MIXED)
        k_kadj<true><<<(n + TPB - 1) / TPB, TPB, 0, st>>>(n, ctx->c, ctx->s4, ctx->p4, ctx->perm, ctx->km, ctx->kv,
                                                           ctx->cis, ctx->rho, ctx->tau, ctx->vs, ctx->gq_own, ctx->gq_tr, dEdq,
                                                           dLdq);
    else
        k_kadj<false><<<(n + TPB - 1) / TPB, TPB, 0, st>>>(n, ctx->c, ctx->s4, ctx->p4, ctx->perm, ctx->km, ctx->kv,
                                                            ctx->cis, ctx->rho, ctx->tau, ctx->vs, ctx->gq_own, ctx->gq_tr, dEdq,
                                                            dLdq);
    prof_end(ctx, RBE_K_KFORCE, st);
}
