// rbe_internal.cuh -- shared declarations of the IRBE CUDA library (sm_103a).
//
// Data layout in HBM (all device buffers owned by rbe_ctx, sized for n_cap
// atoms and grown on demand):
//   sorted order = atoms ordered by (canonical cell, fixed-point x, caller
//   index), built by a counting sort each step (cells of edge L/floor(L/r_c),
//   Sec. 2.3).
//   s4   [n]  uint4   fixed-point (sx, sy, sz) and q as FP32 bits   (16 B/atom)
//   f4   [n]  float4  FP32 wrapped (x, y, z) and q                 (16 B/atom)
//   p4   [n]  double4_32a wrapped (x, y, z) and q in FP64              (32 B/atom)
//   tm   [n]  int2    (type, mol)                                   (8 B/atom)
//   perm [n]  int     sorted index -> caller index
//   F_real [3n] double core + weighted shell force, sorted order
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rbe.h"

#define RBE_MAXT 16
#ifndef RBE_WARPS_RBL
#define RBE_WARPS_RBL 8          // warps per block of the pair kernel
#endif
#ifndef RBE_BLOCKS_RBL
#define RBE_BLOCKS_RBL 2         // resident blocks per SM the pair kernel is sized for
#endif
#ifndef RBE_OVERLAP_KSPACE
// 1: a force evaluation runs the k sampling and the structure factors on an
// auxiliary stream beside the pair kernel (they are independent until the
// finalisation); 0: everything on the caller's stream
#define RBE_OVERLAP_KSPACE 1
#endif
#ifndef RBE_BLOCKS_STORED
// resident blocks per SM of the stored-list (Verlet skin) pair kernel: it
// stages no stencil, so three blocks fit in shared memory; its register
// budget then drops to 80 (a few spills), which the extra resident warps
// repay (measured on the 1.2M-atom water box at a 1 A skin: 3.45 -> 3.13 ms)
#define RBE_BLOCKS_STORED 3
#endif
#define RBE_NPART_RBL 12         // Ec, Elj, Ex, W[6], Fsum[3]
#define RBE_FIN_CHUNKS 64        // chunks of the pair kernel's block partials in the finalisation
#define RBE_NPART_Q 3            // sum q^2, sum q, sum |q|
#define RBE_RBL_PAIR_CARVE 416   // words of the per-warp shell buffer the two-atom pair path uses beyond a core list

// Device status block of a context: word 0 holds the status bits below;
// words 1 and 2 the largest core and shell counts of lists that overflowed
// their capacity (what a retry needs); word 3 the first velocity-Verlet
// launch of rbe_step that found a latched error and stopped (2k for the
// first half kick and drift of step k, 2k + 1 for its second half kick; -1:
// none); word 4 the largest stored list (Verlet skin) that overflowed
#define RBE_STW_NEED_CORE  1
#define RBE_STW_NEED_SHELL 2
#define RBE_STW_HALT       3
#define RBE_STW_NEED_LIST  4
#define RBE_STW_WORDS      5

// status bits latched on the device
#define RBE_ST_OVERLAP   1
#define RBE_ST_CAPACITY  2
#define RBE_ST_NONNEUTRAL 4
#define RBE_ST_NONFINITE 8
#define RBE_ST_KSAMPLE   16
#define RBE_ST_BADTYPE   32
#define RBE_ST_STAGE     64   // a shared-memory staging copy did not complete in time

struct RbeConsts {
    double L, invL, alpha, sqrt_alpha, two_sqrt_alpha_over_sqrt_pi, k_e;
    double r_c, r_s;
    double S;             // H^3 - 1
    double kcoef;         // (S/P) 4 pi k_e / V  (c_l = kcoef / |k_l|^2)
    float Lfix;           // L * 2^-32 (fixed-point unit in length, FP32)
    uint64_t Rc2, Rs2;    // squared radii in fixed-point units
    float rs_frac2;       // (r_s/L)^2 * (1 + 1e-5), for conservative culling
    int n_cell, reach;
    int p, P;
    uint64_t seed;
    int M;                // k truncation
    int ntypes;
    int shift_lj;
    int shell_mode;       // 0: batch without replacement (Floyd), 1: with replacement
    int kpool;            // 0: fresh k draws each step, K > 0: draws from a pool of K
};

// Geometry of the RBL kernel's work units and of its FP32 classification
// prefilter (rbe_api.cu derives it from the box, the cutoffs and the density).
struct RblGeom {
    int G;                 // cells per work unit along x
    int cells_per_row;     // staged cells per stencil row (G + 2R, or n_cell for small boxes)
    int nrows;             // stencil rows of a unit
    int cap_stage;         // staged atoms that fit in shared memory
    int small;             // 1 when the stencil covers the whole box (2R+1 >= n_cell)
    float rc2_lo, rc2_hi;  // r_c^2 minus / plus the FP32 rounding bound (A^2), rounded outward
    float rs2_lo, rs2_hi;  // same for r_s^2
    float tiny2;           // below this squared distance the exact test decides
};

// LJ pair table (device): c12 = 4 eps sig^12, c6 = 4 eps sig^6, shift; for
// the adjoint also the mixed eps_ab, sigma_ab and the derivatives of the
// energy shift with respect to them
struct RbeLJ {
    double c12[RBE_MAXT * RBE_MAXT];
    double c6[RBE_MAXT * RBE_MAXT];
    double shift[RBE_MAXT * RBE_MAXT];
    double eps[RBE_MAXT * RBE_MAXT];
    double sig[RBE_MAXT * RBE_MAXT];
    double dshift_de[RBE_MAXT * RBE_MAXT];
    double dshift_ds[RBE_MAXT * RBE_MAXT];
    double rc2[RBE_MAXT * RBE_MAXT];      // squared LJ cutoff of the pair (huge: no cut below r_s)
};

struct rbe_ctx {
    RbeConsts c;
    int precision;
    int debug, dbg_cap_core;
    int user_core_cap, user_shell_cap;
    int core_cap, shell_cap;
    int profiling;
    double eps[RBE_MAXT], sigma[RBE_MAXT];
    double lj_rc_factor;  // LJ of pair (a, b) cut at min(f sigma_ab, r_s) when f > 0
    int kpool_burn;       // burn-in of the k pool's Metropolis-Hastings chains
    int kpool_dirty;
    int4* kpool_buf;      // [kpool] pool of k samples (device)
    double lang_kT, lang_tau;   // Langevin thermostat (tau <= 0: off)
    double* F_lang;       // [3n] Langevin force, caller order
    size_t F_lang_cap;
    uint64_t lang_step;   // step whose Langevin force F_lang holds (valid if lang_valid)
    int lang_valid, lang_n;
    // water bonds
    int n_wmol;
    double kb, r0, kth, th0;
    char err[512];
    int device;
    // device buffers
    int n_cap;
    long ncells;
    uint4* s4;
    float4* f4;
    double4_32a* p4;
    int2* tm;
    // per-atom records in caller order, written by the quantisation and
    // permuted into s4, f4, p4, tm by the gather: the codes and FP32 charge,
    // the wrapped FP64 position and charge, (type, molecule)
    uint4* rec_s4;
    double4_32a* rec_p4;
    int2* rec_tm;
    // auxiliary stream of the Fourier-space kernels and its fork/join events
    // (created on first use)
    cudaStream_t st_aux;
    cudaEvent_t ev_fork, ev_join;
    int* perm;
    int* cell_of;
    int* slot;
    uint32_t* sx_of;     // [n] fixed-point x code, caller order (in-cell sort key)
    unsigned long long* skey;   // [n] in-cell sort keys (x code << 32 | index), cell ranges
    int* cell_count;     // [ncells + 1]
    int* cell_start;     // [ncells + 1]
    int* scan_tmp;       // [scan tiles] tile sums / offsets of the cell scan
    double* F_real;      // [3n] sorted (FP32 [3n] on the mixed path)
    double* F_bond;      // [3n] caller order
    double* part_rbl;    // [grid_rbl * 12]
    double* fin_part;    // [RBE_FIN_CHUNKS * 12] chunk sums of part_rbl
    double* part_q;      // [grid_q * 3]
    double* part_bond;   // [grid_bond]
    int grid_rbl, grid_q, grid_rho, grid_bond;
    uint64_t* kT;        // [2M+1] inverse-CDF thresholds
    int4* km;            // [P] m
    double4_32a* kv;         // [P] kx, ky, kz, c_l
    double2* rho_part;   // [grid_rho * P]
    double2* cis;        // [65536] e^{2 pi i j / 65536}: FP64 phase table
    double2* rho;        // [P]
    double* totals;      // [32]: E[6], W[6], corr[3], spare
    int* status;         // [RBE_STW_WORDS] status bits, needed capacities, halt code
    long long halt_step; // step whose force evaluation stopped the last rbe_step (-1: none)
    int retrying;        // rbe_forces is re-running a call after a list overflow
    RbeLJ* lj;           // device copy
    int lj_dirty;
    // debug
    int* dbg_ncore;
    int* dbg_nshell;
    int* dbg_core;
    int* dbg_batch;
    int* dbg_unstaged;       // debug [2]: pair-kernel units read from global memory, passes walked range by range
    int dbg_n_cap;
    // host staging for host-pointer calls
    double* h_pos; double* h_q; int* h_type; int* h_mol; double* h_F;
    int h_cap;
    double* ke_part;     // [grid_q] kinetic energy partials (rbe_step)
    // adjoint buffers (rbe_adjoint)
    double* vs;          // [3n] upstream force gradient, sorted order
    double* gq_own;      // [2n] dE/dq, dL/dq from the atom's own pairs (sorted)
    double* gq_tr;       // [2n] same from the pairs of other atoms (sorted)
    double* part_lj;     // [grid_rbl * 4 * nt2] LJ pair-parameter partials
    double* part_v;      // [grid_q * 3] partial sums of the upstream gradient
    double2* tau_part;   // [grid_rho * P]
    double2* tau;        // [P]
    // profiling
    void* prof;          // std::vector of event records (C++ side)
    double prof_ms[RBE_NKERNELS];
    int64_t prof_n[RBE_NKERNELS];
    int last_launches;
    int n_sm, last_n, last_precision;
    int tune_apu;        // target atoms per RBL work unit (0: 48)
    int tune_ups;        // RBL units per slot (0: about 3, at least one wave of resident blocks)
    RblGeom rbl;
    // Verlet skin (stored lists; skin <= 0: off)
    double skin;
    RbeConsts skin_c;     // constants of the list build: both radii r_s + skin, its stencil reach
    RblGeom skin_g;       // work-unit geometry of the list build
    int skin_vcap;        // entries per stored list
    int skin_vcap_min;    // lower bound after an overflow
    int skin_grid_build;  // slots of the list build
    int skin_valid, skin_n;
    long long skin_rebuilds;
    uint64_t skin_D2;     // floor((skin/2 2^32/L)^2): the rebuild threshold
    int* vlist;           // [n * skin_vcap] stored lists (sorted indices of the rebuild)
    int* vcnt;            // [n]
    uint4* sb;            // [n] fixed-point codes at the rebuild, sorted order
    int* inv_perm;        // [n] caller index -> sorted index of the rebuild
    int* skin_moved;      // [1] set when an atom moved more than skin/2 since the rebuild
    size_t skin_cap[5];
    size_t cap_atoms[28];
    size_t cap_adj[8];
};

// ---------------------------------------------------------------------------
// Batched execution: many independent systems ("replicas") stepped together,
// every stage one launch over all replicas.  Each replica keeps its own
// rbe_ctx (buffers, constants, grids); the batched kernels find their replica
// from per-stage block offsets and read its view from a device array.
// ---------------------------------------------------------------------------
struct RepDev {
    int n, nmol, n_bonded_atoms;
    long ncells;
    int grid_q, grid_rho, grid_rbl, grid_bond, rho_chunk;
    double kb, r0, kth, th0;
    double dt, accel;
    RbeConsts c;
    // caller arrays (device, caller order)
    double* pos;
    double* vel;
    const double* mass;
    const double* q;
    const int32_t* type;
    const int32_t* mol;
    double* F;
    // context buffers
    int* cell_count;
    int* cell_start;
    int* cell_of;
    int* slot;
    uint32_t* sx_of;
    unsigned long long* skey;
    int* perm;
    uint4* s4;
    float4* f4;
    double4_32a* p4;
    int2* tm;
    uint4* rec_s4;
    double4_32a* rec_p4;
    int2* rec_tm;
    double* part_q;
    double* part_rbl;
    double* part_bond;
    double* ke_part;
    const uint64_t* kT;
    int4* km;
    double4_32a* kv;
    double2* rho_part;
    double2* rho;
    double* totals;
    double* F_real;
    double* F_bond;
    int* status;
    const int4* kpool;
    const double2* cis;
    double* FL;               // Langevin force [3n] (null: thermostat off)
    double lang_c1, lang_c2;  // accel tau, 24 kT / (accel tau dt)
};

// Device control block of a batch: the MD step the batched kernels use, the
// energy trace and the head of the pair kernel's work queue.
struct BatchCtl {
    unsigned long long step, step0;
    double* trace;         // [nrep][nsteps][2] or null
    int nsteps;
    int rbl_next;
};

// Stages of a batched step, each with its own per-replica block counts.
enum { BK_CELLS = 0, BK_ATOMS, BK_Q, BK_KS, BK_RHO, BK_BOND, BK_REP, BK_RS, BK_COUNT };

struct BatchPlan {
    int nrep;
    int precision;
    const RepDev* rep;               // [nrep] device
    const int* off[BK_COUNT];        // [nrep + 1] device, exclusive prefix sums of block counts
    int total[BK_COUNT];             // blocks of each batched launch
    BatchCtl* ctl;                   // device
    int rho_threads;                 // threads of the batched rho kernel (max over replicas)
    // persistent pair kernel
    const void* rbl_args;            // [nrep] device, RblArgs (k_rbl.cu)
    const int2* tasks;               // [ntasks] device, (replica, slot) by decreasing cost
    int ntasks;
    int rbl_grid, rbl_smem;
    int rbl_persistent;              // 1: rbl_grid resident blocks over the queue; 0: one block per task
};

// Replica that owns block b of a batched launch whose per-replica block counts
// have the exclusive prefix sums off[0..nrep] (off[0] = 0 <= b < off[nrep]),
// b's index within that replica's grid and the size of that grid.
__device__ __forceinline__ int rep_of_block(const int* __restrict__ off, int nrep, int b, int& local, int& count)
{
    int lo = 0, hi = nrep;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid;
    }
    local = b - off[lo];
    count = off[lo + 1] - off[lo];
    return lo;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 64x64
// multiplies with the published multipliers and Weyl key increments.
__device__ __forceinline__ void philox4x64_10(uint64_t x0, uint64_t x1, uint64_t x2, uint64_t x3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
        uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
        uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Fractional coordinate and 32-bit fixed-point code of x (identical IEEE
// operations on host and device: the products are explicitly rounded so that
// no multiply-add contraction changes them).
__device__ __forceinline__ void wrap_fixed(double x, double invL, double L, double& xw, uint32_t& s)
{
    double t = __dmul_rn(x, invL);
    double f = __dsub_rn(t, floor(t));
    if (f >= 1.0) f = 0.0;
    // s = floor(f 2^32) for 0 <= f < 1, from the bits of f: f 2^32 is exact,
    // so its integer part is the 53-bit significand shifted right by 20 - e
    // (e = f's exponent <= -1; 0 once the shift reaches 64, which covers f = 0
    // and subnormal f).  Integer instructions instead of an FP64 multiply and
    // conversion: GB300's FP64 pipe is the bound of this arithmetic.
    const unsigned long long u = (unsigned long long)__double_as_longlong(f);
    const int sh = 20 - ((int)((u >> 52) & 0x7FFull) - 1023);
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    s = sh < 64 ? (uint32_t)(m >> sh) : 0u;
    xw = __dmul_rn(f, L);
}

__device__ __forceinline__ uint32_t cell_of_fixed(uint32_t s, int n_cell)
{
    return (uint32_t)(((uint64_t)s * (uint64_t)n_cell) >> 32);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void latch_status(int* status, int bit) { atomicOr(status, bit); }

// Bulk asynchronous copies (TMA, non-tensor form) from global to shared
// memory, completing on a shared-memory mbarrier: the barrier's arrival count
// is 1 (the thread that posts the expected bytes), each copy decrements its
// transaction count by the bytes it wrote, and the phase completes when both
// reach zero.  Addresses 16-byte aligned, sizes multiples of 16.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* m)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Waits for the phase of the given parity to complete, giving up after
// `limit` polls (each poll may suspend the thread for a short while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, uint32_t parity, int limit)
{
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m)
{
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}
// Asynchronous 16-byte global -> shared copies (both addresses 16-byte
// aligned); a thread sees its own copies after cp_async_wait, other threads'
// after that and a barrier.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most N of this thread's committed groups are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// Orders this thread's earlier generic-proxy accesses to shared memory before
// its later async-proxy ones (a bulk copy into memory that was just written).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// floor(u * n / 2^64) for n < 2^32: a uniform integer in [0, n) from a 64-bit word.
__device__ __forceinline__ uint32_t uniform_below(uint64_t u, uint32_t n)
{
    uint64_t lo = (uint64_t)(uint32_t)u * n;
    uint64_t hi = (uint64_t)(uint32_t)(u >> 32) * n;
    return (uint32_t)((hi + (lo >> 32)) >> 32);
}

// ---------------------------------------------------------------------------
// kernel launchers (each returns the number of kernels enqueued)
// ---------------------------------------------------------------------------
struct Launch;   // profiling helper (rbe_api.cu)
void prof_begin(rbe_ctx* ctx, int kid, cudaStream_t st);
void prof_end(rbe_ctx* ctx, int kid, cudaStream_t st);

// cells / sort (k_cells.cu)
void launch_quantize_count(rbe_ctx* ctx, int n, const double* pos, const double* q, const int32_t* type,
                           const int32_t* mol, cudaStream_t st);
void launch_scan(rbe_ctx* ctx, cudaStream_t st);
long scan_tiles(long ncells);
void launch_scatter_sort_gather(rbe_ctx* ctx, int n, cudaStream_t st);
// pair kernel (k_rbl.cu)
void launch_rbl(rbe_ctx* ctx, int n, uint64_t step, cudaStream_t st, bool adjoint = false);
// adjoint (k_kspace.cu)
void launch_adj_prep(rbe_ctx* ctx, int n, const double* gF, cudaStream_t st);
void launch_adj_final(rbe_ctx* ctx, int n, double* dEdq, double* dLdq, cudaStream_t st);
// Fourier part and finalisation (k_kspace.cu)
void launch_ksample(rbe_ctx* ctx, uint64_t step, cudaStream_t st);
// Metropolis-Hastings pool of k samples from host-made tables (k_kspace.cu)
void launch_kpool_build(rbe_ctx* ctx, const double* w, const double* q, const uint64_t* Tq, int M, cudaStream_t st);
void launch_rho(rbe_ctx* ctx, int n, cudaStream_t st);
void launch_cis_table(double2* tab, cudaStream_t st);
void launch_bonded(rbe_ctx* ctx, int n, const double* pos, cudaStream_t st);
void launch_finalize(rbe_ctx* ctx, int n, cudaStream_t st);
void launch_kforce(rbe_ctx* ctx, int n, double* F, cudaStream_t st);
void launch_vv_kick_drift(rbe_ctx* ctx, int n, double* pos, double* vel, const double* mass,
                          const double* F, const double* FL, double dt, double accel, int drift, int code,
                          cudaStream_t st);
void launch_langevin(rbe_ctx* ctx, int n, const double* vel, const double* mass, uint64_t s, double dt,
                     double accel, cudaStream_t st);
void launch_langevin_batch(const BatchPlan& bp, const int* mask, cudaStream_t st);
void launch_ke_trace(rbe_ctx* ctx, int n, const double* vel, const double* mass, double accel,
                     double* trace_slot, cudaStream_t st);
int rbl_smem_bytes(const rbe_ctx* ctx);
int rbl_smem_target();
// validation and device set-up of one context for n atoms (rbe_api.cu)
int ctx_prepare(rbe_ctx* ctx, int n);
// Langevin force buffer of a context for n atoms (rbe_api.cu)
int ctx_grow_lang(rbe_ctx* ctx, int n);
// batched stages (one launch each over all replicas of a plan)
void launch_cells_batch(const BatchPlan& bp, cudaStream_t st);
void launch_kspace_pre_batch(const BatchPlan& bp, cudaStream_t st);
void launch_kspace_post_batch(const BatchPlan& bp, cudaStream_t st);
void launch_vv_batch(const BatchPlan& bp, int drift, cudaStream_t st);
void launch_ke_trace_batch(const BatchPlan& bp, cudaStream_t st);
// op 0: set step = step0 (and the trace); 1: advance one step; 2: reset the work queue only
void launch_ctl_batch(const BatchPlan& bp, int op, unsigned long long step0, double* trace, int nsteps,
                      cudaStream_t st);
void launch_rbl_batch(const BatchPlan& bp, cudaStream_t st);
size_t rbl_args_bytes();
void rbl_fill_args(const rbe_ctx* ctx, int n, void* out);
int rbl_max_blocks_per_sm(int precision, int smem);
long rbl_units(const rbe_ctx* ctx);
int rbl_blocks_per_sm(const rbe_ctx* ctx);
// Verlet-skin variant (stored lists)
void launch_skin_gather(rbe_ctx* ctx, int n, const double* pos, const double* q, const int32_t* type,
                        const int32_t* mol, cudaStream_t st);
void launch_skin_mark(rbe_ctx* ctx, int n, cudaStream_t st);
void launch_rbl_build(rbe_ctx* ctx, int n, cudaStream_t st);
void launch_rbl_stored(rbe_ctx* ctx, int n, uint64_t step, cudaStream_t st);
int rbl_build_smem_bytes(const rbe_ctx* ctx);
long rbl_build_units(const rbe_ctx* ctx);
