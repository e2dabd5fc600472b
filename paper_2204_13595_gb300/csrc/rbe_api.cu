// rbe_api.cu -- host side of the C ABI declared in include/rbe.h: context,
// parameter derivation, device memory, the launch sequence of one force step
// and the velocity-Verlet driver.
//
// Launch sequence of rbe_forces on one stream (Algorithm 1, force steps):
//   quantize+count -> scan -> scatter/sort/gather   (cell list, Sec. 2.3)
//   k sample -> rho partials -> rho sum             (RBE, Eqs. (2.4), (2.8))
//   RBL pair kernel                                 (Eqs. (2.10)-(2.11))
//   [bonded water]                                  (integration force field)
//   finalize: energies, virial, F^corr              (Eqs. (2.3), (2.12))
//   k-space force + combination                     (Eqs. (2.9), (2.13))
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rbe_internal.cuh"

namespace {

const double PI = 3.14159265358979323846;

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};
struct ProfState {
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t pending_a = nullptr;
};

int set_err(rbe_ctx* ctx, int code, const char* fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CUDA_TRY(ctx, call)                                                                         \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return set_err(ctx, RBE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

// Inverse-CDF thresholds of the per-axis discrete Gaussian
// w_m = exp(-pi^2 m^2 / (alpha L^2)), |m| <= M (reading of Eqs. (2.7)-(2.8)):
// T[m+M] = floor(2^64 * sum_{j<=m} w_j / H), saturating at 2^64-1.
int k_truncation(double alpha, double L)
{
    double aL2 = alpha * L * L;
    return (int)ceil(sqrt(aL2 * 64.0 * log(2.0)) / PI);
}

double k_thresholds(double alpha, double L, int M, uint64_t* T)
{
    double aL2 = alpha * L * L;
    double c = PI * PI / aL2;
    double H = 0.0;
    for (int m = -M; m <= M; ++m) H += exp(-c * (double)m * (double)m);
    double acc = 0.0;
    for (int m = -M; m <= M; ++m) {
        acc += exp(-c * (double)m * (double)m);
        double v = (acc / H) * 18446744073709551616.0;
        T[m + M] = (v >= 18446744073709551616.0) ? UINT64_MAX : (uint64_t)v;
    }
    return H;
}

// Tables of the Metropolis-Hastings k pool (Algorithm 1, pool step; Sec. 2.2
// sampling text): target w_m = exp(-pi^2 m^2/(alpha L^2)) and proposal
// q_m = P(round(X) = m), X ~ N(0, s^2), s^2 = alpha L^2/(2 pi^2), on |m| <= M,
// with the 64-bit inverse-CDF thresholds of q (normalised on |m| <= M).
void mh_tables(double alpha, double L, int M, double* w, double* q, uint64_t* Tq)
{
    const double aL2 = alpha * L * L;
    const double c = PI * PI / aL2;
    const double sd = sqrt(aL2 / (2.0 * PI * PI));
    const double sq2 = sd * sqrt(2.0);
    double Q = 0.0;
    for (int m = -M; m <= M; ++m) {
        w[m + M] = exp(-c * (double)m * (double)m);
        const double am = fabs((double)m);
        const double lo = (am - 0.5) / sq2, hi = (am + 0.5) / sq2;
        const double qm = (m == 0) ? erf(0.5 / sq2) : 0.5 * (erfc(lo) - erfc(hi));
        q[m + M] = qm;
        Q += qm;
    }
    double acc = 0.0;
    for (int m = -M; m <= M; ++m) {
        acc += q[m + M];
        const double v = (acc / Q) * 18446744073709551616.0;
        Tq[m + M] = (v >= 18446744073709551616.0) ? UINT64_MAX : (uint64_t)v;
    }
}

uint64_t radius2_fixed(double r, double L)
{
    double invL = 1.0 / L;
    double a = (r * invL) * 4294967296.0;
    return (uint64_t)(a * a);
}

void refresh_consts(rbe_ctx* ctx)
{
    RbeConsts& c = ctx->c;
    c.invL = 1.0 / c.L;
    c.sqrt_alpha = sqrt(c.alpha);
    c.two_sqrt_alpha_over_sqrt_pi = 2.0 * sqrt(c.alpha) / sqrt(PI);
    double V = c.L * c.L * c.L;
    c.kcoef = (c.S / (double)c.P) * 4.0 * PI * c.k_e / V;
    c.Lfix = (float)(c.L * 2.3283064365386963e-10);
}

void free_dev(rbe_ctx* ctx)
{
    void* ptrs[] = {ctx->cis, ctx->skey, ctx->scan_tmp, ctx->sx_of, ctx->F_lang, ctx->kpool_buf, ctx->s4, ctx->f4, ctx->p4, ctx->tm, ctx->rec_s4, ctx->rec_p4, ctx->rec_tm, ctx->fin_part, ctx->perm, ctx->cell_of, ctx->slot, ctx->cell_count, ctx->cell_start,
                    ctx->F_real, ctx->F_bond, ctx->part_rbl, ctx->part_q, ctx->part_bond, ctx->kT, ctx->km, ctx->kv,
                    ctx->rho_part, ctx->rho, ctx->totals, ctx->status, ctx->lj, ctx->dbg_ncore, ctx->dbg_nshell,
                    ctx->dbg_core, ctx->dbg_batch, ctx->dbg_unstaged, ctx->h_pos, ctx->h_q, ctx->h_type, ctx->h_mol, ctx->h_F,
                    ctx->ke_part, ctx->vs, ctx->gq_own, ctx->gq_tr, ctx->part_lj, ctx->part_v, ctx->tau_part,
                    ctx->tau, ctx->vlist, ctx->vcnt, ctx->sb, ctx->inv_perm, ctx->skin_moved};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ctx->vlist = nullptr; ctx->vcnt = nullptr; ctx->sb = nullptr; ctx->inv_perm = nullptr; ctx->skin_moved = nullptr;
    for (int k = 0; k < 5; ++k) ctx->skin_cap[k] = 0;
    ctx->skin_valid = 0;
    ctx->s4 = nullptr; ctx->f4 = nullptr; ctx->p4 = nullptr; ctx->tm = nullptr; ctx->perm = nullptr; ctx->cell_of = nullptr;
    ctx->rec_s4 = nullptr; ctx->rec_p4 = nullptr; ctx->rec_tm = nullptr; ctx->fin_part = nullptr;
    ctx->slot = nullptr; ctx->cell_count = nullptr; ctx->cell_start = nullptr; ctx->F_real = nullptr;
    ctx->F_bond = nullptr; ctx->part_rbl = nullptr; ctx->part_q = nullptr; ctx->part_bond = nullptr;
    ctx->kT = nullptr; ctx->km = nullptr; ctx->kv = nullptr; ctx->rho_part = nullptr; ctx->rho = nullptr;
    ctx->totals = nullptr; ctx->status = nullptr; ctx->lj = nullptr; ctx->dbg_ncore = nullptr;
    ctx->dbg_nshell = nullptr; ctx->dbg_core = nullptr; ctx->dbg_batch = nullptr; ctx->dbg_unstaged = nullptr;
    ctx->h_pos = nullptr;
    ctx->h_q = nullptr; ctx->h_type = nullptr; ctx->h_mol = nullptr; ctx->h_F = nullptr; ctx->ke_part = nullptr;
    ctx->vs = nullptr; ctx->gq_own = nullptr; ctx->gq_tr = nullptr; ctx->part_lj = nullptr; ctx->part_v = nullptr;
    ctx->tau_part = nullptr; ctx->tau = nullptr; ctx->kpool_buf = nullptr; ctx->kpool_dirty = 1;
    ctx->F_lang = nullptr; ctx->F_lang_cap = 0; ctx->sx_of = nullptr; ctx->scan_tmp = nullptr; ctx->skey = nullptr; ctx->cis = nullptr;
    ctx->n_cap = 0; ctx->dbg_n_cap = 0; ctx->h_cap = 0;
    for (int k = 0; k < 28; ++k) ctx->cap_atoms[k] = 0;
    for (int k = 0; k < 8; ++k) ctx->cap_adj[k] = 0;
}

template <typename T>
int dev_alloc(rbe_ctx* ctx, T** p, size_t count)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        return set_err(ctx, RBE_ENOMEM, "cudaMalloc of %zu bytes failed: %s", sizeof(T) * count, cudaGetErrorString(e));
    }
    return RBE_OK;
}

int round32(double x) { return ((int)ceil(x) + 31) / 32 * 32; }

// Capacities of the per-warp core and shell buffers from the density:
// twice the mean count plus six standard deviations plus a margin; the shell
// buffer also holds what the pair kernel's two-atom path keeps beyond a
// second core list.
void auto_caps(rbe_ctx* ctx, int n)
{
    double rho = (double)n / (ctx->c.L * ctx->c.L * ctx->c.L);
    double rc = ctx->c.r_c, rs = ctx->c.r_s;
    double mc = 4.0 / 3.0 * PI * rc * rc * rc * rho;
    double ms = 4.0 / 3.0 * PI * (rs * rs * rs - rc * rc * rc) * rho;
    int cc = ctx->user_core_cap > 0 ? ctx->user_core_cap : round32(2.0 * mc + 6.0 * sqrt(mc) + 32.0);
    int sc = ctx->user_shell_cap > 0 ? ctx->user_shell_cap : round32(2.0 * ms + 6.0 * sqrt(ms) + 32.0);
    ctx->core_cap = (cc + 31) / 32 * 32;
    ctx->shell_cap = (sc + 31) / 32 * 32;
    if (ctx->user_shell_cap <= 0 && ctx->shell_cap < ctx->core_cap + RBE_RBL_PAIR_CARVE)
        ctx->shell_cap = (ctx->core_cap + RBE_RBL_PAIR_CARVE + 31) / 32 * 32;
}

// Work-unit geometry of the RBL kernel and the rounding bound of its FP32
// classification prefilter.  Positions are FP32 copies of the wrapped FP64
// coordinates (error <= L 2^-24 each, plus L 2^-32 from the fixed-point code),
// so each displacement component is off by at most da = 3 L 2^-23 + r 2^-24
// and r^2 by at most 2 sqrt(3) r da + 3 da^2 + 3 r^2 2^-23; the bands are four
// times that bound wide, and inside them the exact integer test decides.
// Work units of one form of the pair kernel (g, with the stencil reach of c)
// for n atoms: G cells per unit, staging capacity, bands of the FP32
// prefilter around the squared radii rc and rs; smem_of gives the form's
// shared memory for the current g.
void unit_geometry(rbe_ctx* ctx, int n, const RbeConsts& c, double rc, double rs, RblGeom& g,
                   int (*smem_of)(const rbe_ctx*))
{
    const int nc = c.n_cell, R = c.reach;
    g.small = (2 * R + 1 >= nc) ? 1 : 0;
    double apc = (double)n / ((double)nc * nc * nc);
    int naxis = g.small ? nc : 2 * R + 1;
    g.nrows = naxis * naxis;
    // shared memory per block: two resident blocks per SM
    const int target = rbl_smem_target();
    const double apu = ctx->tune_apu > 0 ? (double)ctx->tune_apu : 64.0;
    int G = (int)lrint(apu / (apc > 1e-9 ? apc : 1e-9));
    G = G < 1 ? 1 : (G > nc ? nc : G);
    for (;; --G) {
        g.G = G;
        g.cells_per_row = g.small ? nc : G + 2 * R;
        double region = g.small ? (double)n : (double)g.cells_per_row * g.nrows * apc;
        // the mean region plus eight Poisson standard deviations and a
        // margin; a unit beyond it reads global memory instead (correct,
        // slower: only strongly inhomogeneous systems get there)
        int cap = (int)ceil(region + 8.0 * sqrt(region) + 256.0);
        cap = (cap + 63) / 64 * 64;
        const int maxcap = (96 * 1024) / 16;
        g.cap_stage = cap < maxcap ? cap : maxcap;
        if (G == 1 || smem_of(ctx) <= target) break;
    }
    auto bound = [&](double r) {
        double da = 3.0 * c.L * 1.1920928955078125e-07 + r * 5.9604644775390625e-08;
        return 4.0 * (2.0 * sqrt(3.0) * r * da + 3.0 * da * da + 3.0 * r * r * 1.1920928955078125e-07);
    };
    double rc2 = rc * rc, rs2 = rs * rs;
    // thresholds rounded outward: the FP32 value of a band's lower edge is
    // at most, and of its upper edge at least, the exact edge
    g.rc2_lo = nextafterf((float)(rc2 - bound(rc)), 0.0f);
    g.rc2_hi = nextafterf((float)(rc2 + bound(rc)), 3.0e38f);
    g.rs2_lo = nextafterf((float)(rs2 - bound(rs)), 0.0f);
    g.rs2_hi = nextafterf((float)(rs2 + bound(rs)), 3.0e38f);
    g.tiny2 = nextafterf((float)(1e-6 * c.r_c * c.r_c + bound(0.0)), 3.0e38f);
}

void rbl_geometry(rbe_ctx* ctx, int n)
{
    unit_geometry(ctx, n, ctx->c, ctx->c.r_c, ctx->c.r_s, ctx->rbl, rbl_smem_bytes);
}

// Verlet skin: constants, geometry and capacity of the list build (both
// radii r_v = r_s + skin: every member of the stored list counts as "core"),
// and the rebuild threshold floor((skin/2 2^32/L)^2).
void skin_geometry(rbe_ctx* ctx, int n)
{
    const double rv = ctx->c.r_s + ctx->skin;
    RbeConsts& b = ctx->skin_c;
    b = ctx->c;
    b.r_s = rv;
    b.Rc2 = b.Rs2 = radius2_fixed(rv, ctx->c.L);
    b.reach = (int)floor(rv * (double)ctx->c.n_cell / ctx->c.L) + 1;
    b.rs_frac2 = (float)((rv / ctx->c.L) * (rv / ctx->c.L) * (1.0 + 1e-5));
    ctx->skin_D2 = radius2_fixed(0.5 * ctx->skin, ctx->c.L);
    const double rho = (double)n / (ctx->c.L * ctx->c.L * ctx->c.L);
    const double mv = 4.0 / 3.0 * PI * rv * rv * rv * rho;
    ctx->skin_vcap = round32(1.25 * mv + 8.0 * sqrt(mv) + 64.0);
    if (ctx->skin_vcap < ctx->skin_vcap_min) ctx->skin_vcap = (ctx->skin_vcap_min + 31) / 32 * 32;
    unit_geometry(ctx, n, b, rv, rv, ctx->skin_g, rbl_build_smem_bytes);
    // no shell in the build: the shell band is the core band's upper edge
    ctx->skin_g.rs2_lo = ctx->skin_g.rs2_hi = ctx->skin_g.rc2_hi;
    const long units = rbl_build_units(ctx);
    long gb = (units + 2) / 3;
    const long wave = 2L * ctx->n_sm;
    if (gb < wave) gb = wave;
    if (gb > units) gb = units;
    ctx->skin_grid_build = (int)(gb < 1 ? 1 : gb);
}

// Reallocates *p only when `count` exceeds the recorded capacity *cap.
template <typename T>
int grow(rbe_ctx* ctx, T** p, size_t* cap, size_t count)
{
    if (*p && count <= *cap) return RBE_OK;
    int rc = dev_alloc(ctx, p, count);
    *cap = rc ? 0 : (count == 0 ? 1 : count);
    return rc;
}

int ensure(rbe_ctx* ctx, int n)
{
    int dev = 0;
    CUDA_TRY(ctx, cudaGetDevice(&dev));
    if (ctx->device >= 0 && dev != ctx->device)
        return set_err(ctx, RBE_EINVAL, "context was created on device %d, current device is %d", ctx->device, dev);
    bool first = ctx->device < 0;
    ctx->device = dev;
    int rc;
    if (first) {
        CUDA_TRY(ctx, cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev));
        // fixed-size buffers
        int M = ctx->c.M;
        std::vector<uint64_t> T(2 * M + 1);
        k_thresholds(ctx->c.alpha, ctx->c.L, M, T.data());
        if ((rc = dev_alloc(ctx, &ctx->kT, T.size()))) return rc;
        CUDA_TRY(ctx, cudaMemcpy(ctx->kT, T.data(), sizeof(uint64_t) * T.size(), cudaMemcpyHostToDevice));
        if ((rc = dev_alloc(ctx, &ctx->km, ctx->c.P))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->kv, ctx->c.P))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->rho, ctx->c.P))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->cis, 65536))) return rc;
        launch_cis_table(ctx->cis, 0);
        CUDA_TRY(ctx, cudaDeviceSynchronize());
        if ((rc = dev_alloc(ctx, &ctx->totals, 32 + 7 * (size_t)ctx->c.P))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->status, RBE_STW_WORDS))) return rc;
        {
            const int init[RBE_STW_WORDS] = {0, 0, 0, -1, 0};
            CUDA_TRY(ctx, cudaMemcpy(ctx->status, init, sizeof(init), cudaMemcpyHostToDevice));
        }
        CUDA_TRY(ctx, cudaMemset(ctx->totals, 0, sizeof(double) * (32 + 7 * (size_t)ctx->c.P)));
        if ((rc = dev_alloc(ctx, &ctx->lj, 1))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->cell_count, ctx->ncells + 1))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->cell_start, ctx->ncells + 1))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->scan_tmp, (size_t)scan_tiles(ctx->ncells) + 1))) return rc;
        ctx->lj_dirty = 1;
    }
    if (ctx->lj_dirty) {
        RbeLJ h;
        memset(&h, 0, sizeof(h));
        for (int a = 0; a < ctx->c.ntypes; ++a)
            for (int b = 0; b < ctx->c.ntypes; ++b) {
                double e = sqrt(ctx->eps[a] * ctx->eps[b]);          // Berthelot
                double s = 0.5 * (ctx->sigma[a] + ctx->sigma[b]);    // Lorentz
                double s6 = s * s * s * s * s * s;
                h.c12[a * RBE_MAXT + b] = 4.0 * e * s6 * s6;
                h.c6[a * RBE_MAXT + b] = 4.0 * e * s6;
                // LJ cutoff of the pair: min(f sigma_ab, r_s) (f = 2^(1/6) with
                // the shift: the WCA soft sphere); beyond r_s no pair is summed
                double rc = ctx->c.r_s;
                bool cut = false;
                if (ctx->lj_rc_factor > 0.0 && ctx->lj_rc_factor * s < ctx->c.r_s) {
                    rc = ctx->lj_rc_factor * s;
                    cut = true;
                }
                h.rc2[a * RBE_MAXT + b] = cut ? rc * rc : 1.0e300;
                double sr6 = pow(s / rc, 6.0);
                h.shift[a * RBE_MAXT + b] = ctx->c.shift_lj ? 4.0 * e * (sr6 * sr6 - sr6) : 0.0;
                h.eps[a * RBE_MAXT + b] = e;
                h.sig[a * RBE_MAXT + b] = s;
                h.dshift_de[a * RBE_MAXT + b] = ctx->c.shift_lj ? 4.0 * (sr6 * sr6 - sr6) : 0.0;
                // with rc = f sigma the shift does not depend on sigma
                h.dshift_ds[a * RBE_MAXT + b] =
                    (ctx->c.shift_lj && !cut) ? 4.0 * e * (12.0 * sr6 * sr6 - 6.0 * sr6) / s : 0.0;
            }
        CUDA_TRY(ctx, cudaMemcpy(ctx->lj, &h, sizeof(h), cudaMemcpyHostToDevice));
        ctx->lj_dirty = 0;
    }
    if (ctx->c.kpool > 0 && (ctx->kpool_dirty || !ctx->kpool_buf)) {
        // k pool: tables on the host, the chains on the device (set-up, once)
        const int M = ctx->c.M;
        std::vector<double> w(2 * M + 1), q(2 * M + 1);
        std::vector<uint64_t> Tq(2 * M + 1);
        mh_tables(ctx->c.alpha, ctx->c.L, M, w.data(), q.data(), Tq.data());
        double *dw = nullptr, *dq = nullptr;
        uint64_t* dT = nullptr;
        if ((rc = dev_alloc(ctx, &ctx->kpool_buf, (size_t)ctx->c.kpool))) return rc;
        if ((rc = dev_alloc(ctx, &dw, w.size()))) return rc;
        if ((rc = dev_alloc(ctx, &dq, q.size()))) { cudaFree(dw); return rc; }
        if ((rc = dev_alloc(ctx, &dT, Tq.size()))) { cudaFree(dw); cudaFree(dq); return rc; }
        cudaMemcpy(dw, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dq, q.data(), sizeof(double) * q.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dT, Tq.data(), sizeof(uint64_t) * Tq.size(), cudaMemcpyHostToDevice);
        launch_kpool_build(ctx, dw, dq, dT, M, 0);
        cudaError_t e = cudaDeviceSynchronize();
        cudaFree(dw); cudaFree(dq); cudaFree(dT);
        if (e != cudaSuccess) return set_err(ctx, RBE_ECUDA, "k pool build failed: %s", cudaGetErrorString(e));
        ctx->kpool_dirty = 0;
    }
    if (n != ctx->last_n || ctx->precision != ctx->last_precision) {
        auto_caps(ctx, n);
        rbl_geometry(ctx, n);
        if (rbl_smem_bytes(ctx) > 220 * 1024)
            return set_err(ctx, RBE_ECAPACITY, "list capacities (%d core, %d shell) exceed shared memory",
                           ctx->core_cap, ctx->shell_cap);
        // grids (fixed for a given n and device, so every reduction order is fixed)
        int nsm = ctx->n_sm;
        ctx->grid_q = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
        // pair kernel slots (one block each, units round-robin over the
        // slots): ceil(units / tune_ups) when tuned; by default about three
        // units per slot, and at least one full wave of resident blocks
        // (measured on the 1.2M-atom water box: 3-4 units per slot beat a
        // persistent grid of blocks_per_sm x SMs slots by 11%, the hardware
        // block scheduler balancing the uneven unit costs); never more
        // slots than units
        int bps = rbl_blocks_per_sm(ctx);
        long units = rbl_units(ctx);
        const long wave = (long)bps * nsm;
        long g = ctx->tune_ups > 0 ? (units + ctx->tune_ups - 1) / ctx->tune_ups : (units + 2) / 3;
        if (ctx->tune_ups == 0 && g < wave) g = wave;
        if (g > units) g = units;
        ctx->grid_rbl = (int)(g < 1 ? 1 : g);
        // structure-factor blocks (each owns a chunk of atoms for all P k):
        // eight per SM keep the special-function pipe fed (measured at 1.2M
        // atoms: 0.152 ms with two per SM, 0.129 ms with eight, the partial
        // sums' reduction 0.005 ms longer)
        int gr = (n + 255) / 256;
        ctx->grid_rho = gr < 8 * nsm ? gr : 8 * nsm;
        if (ctx->skin > 0.0) {
            skin_geometry(ctx, n);
            if (rbl_build_smem_bytes(ctx) > 220 * 1024)
                return set_err(ctx, RBE_ECAPACITY, "stored-list capacity %d exceeds shared memory", ctx->skin_vcap);
            ctx->skin_valid = 0;
        }
        ctx->last_n = n;
        ctx->last_precision = ctx->precision;
    }
    if (ctx->skin > 0.0) {
        if ((rc = grow(ctx, &ctx->vlist, &ctx->skin_cap[0], (size_t)n * ctx->skin_vcap))) return rc;
        if ((rc = grow(ctx, &ctx->vcnt, &ctx->skin_cap[1], n))) return rc;
        if ((rc = grow(ctx, &ctx->sb, &ctx->skin_cap[2], n))) return rc;
        if ((rc = grow(ctx, &ctx->inv_perm, &ctx->skin_cap[3], n))) return rc;
        if ((rc = grow(ctx, &ctx->skin_moved, &ctx->skin_cap[4], 1))) return rc;
    }
    int gb = ctx->n_wmol > 0 ? (ctx->n_wmol + 255) / 256 : 0;
    ctx->grid_bond = gb < 4 * ctx->n_sm ? gb : 4 * ctx->n_sm;
    if ((rc = grow(ctx, &ctx->s4, &ctx->cap_atoms[0], n))) return rc;
    if ((rc = grow(ctx, &ctx->f4, &ctx->cap_atoms[17], n))) return rc;
    if ((rc = grow(ctx, &ctx->p4, &ctx->cap_atoms[1], n))) return rc;
    if ((rc = grow(ctx, &ctx->tm, &ctx->cap_atoms[2], n))) return rc;
    if ((rc = grow(ctx, &ctx->rec_s4, &ctx->cap_atoms[23], n))) return rc;
    if ((rc = grow(ctx, &ctx->rec_p4, &ctx->cap_atoms[24], n))) return rc;
    if ((rc = grow(ctx, &ctx->rec_tm, &ctx->cap_atoms[25], n))) return rc;
    if ((rc = grow(ctx, &ctx->fin_part, &ctx->cap_atoms[26], (size_t)RBE_FIN_CHUNKS * RBE_NPART_RBL))) return rc;
    if ((rc = grow(ctx, &ctx->perm, &ctx->cap_atoms[3], n))) return rc;
    if ((rc = grow(ctx, &ctx->cell_of, &ctx->cap_atoms[4], n))) return rc;
    if ((rc = grow(ctx, &ctx->slot, &ctx->cap_atoms[5], n))) return rc;
    if ((rc = grow(ctx, &ctx->sx_of, &ctx->cap_atoms[20], n))) return rc;
    if ((rc = grow(ctx, &ctx->skey, &ctx->cap_atoms[21], n))) return rc;
    if ((rc = grow(ctx, &ctx->F_real, &ctx->cap_atoms[6], 3 * (size_t)n))) return rc;
    if ((rc = grow(ctx, &ctx->part_rbl, &ctx->cap_atoms[7], (size_t)ctx->grid_rbl * RBE_NPART_RBL))) return rc;
    if ((rc = grow(ctx, &ctx->part_q, &ctx->cap_atoms[8], (size_t)ctx->grid_q * RBE_NPART_Q))) return rc;
    if ((rc = grow(ctx, &ctx->ke_part, &ctx->cap_atoms[9], (size_t)ctx->grid_q))) return rc;
    if ((rc = grow(ctx, &ctx->part_bond, &ctx->cap_atoms[10], (size_t)(ctx->grid_bond > 0 ? ctx->grid_bond : 1)))) return rc;
    if ((rc = grow(ctx, &ctx->rho_part, &ctx->cap_atoms[11], (size_t)ctx->grid_rho * ctx->c.P))) return rc;
    if (ctx->n_wmol > 0 && (rc = grow(ctx, &ctx->F_bond, &ctx->cap_atoms[12], 9 * (size_t)ctx->n_wmol))) return rc;
    ctx->n_cap = (int)ctx->cap_atoms[0];
    if (ctx->debug) {
        size_t cc = (size_t)(ctx->dbg_cap_core > 0 ? ctx->dbg_cap_core : 1);
        if ((rc = grow(ctx, &ctx->dbg_ncore, &ctx->cap_atoms[13], n))) return rc;
        if ((rc = grow(ctx, &ctx->dbg_nshell, &ctx->cap_atoms[14], n))) return rc;
        if ((rc = grow(ctx, &ctx->dbg_core, &ctx->cap_atoms[15], (size_t)n * cc))) return rc;
        if ((rc = grow(ctx, &ctx->dbg_batch, &ctx->cap_atoms[16], (size_t)n * ctx->c.p))) return rc;
        if ((rc = grow(ctx, &ctx->dbg_unstaged, &ctx->cap_atoms[22], 2))) return rc;
        ctx->dbg_n_cap = n;
    }
    return RBE_OK;
}

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The device address of pinned host memory that the device can read in
// place (page-locked and mapped into the device's address space), else null.
const void* pinned_device_view(const void* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

}  // namespace

int ctx_prepare(rbe_ctx* ctx, int n)
{
    if (n < 1) return set_err(ctx, RBE_EINVAL, "n >= 1 is required");
    if (ctx->n_wmol > 0 && 3 * ctx->n_wmol > n)
        return set_err(ctx, RBE_EINVAL, "water bonds cover %d atoms but n = %d", 3 * ctx->n_wmol, n);
    return ensure(ctx, n);
}

int ctx_grow_lang(rbe_ctx* ctx, int n)
{
    double* old = ctx->F_lang;
    int rc = grow(ctx, &ctx->F_lang, &ctx->F_lang_cap, 3 * (size_t)n);
    if (ctx->F_lang != old) ctx->lang_valid = 0;      // a new buffer holds no force
    return rc;
}

namespace {

// Verlet skin (reading R15): between rebuilds the atoms keep the sorted
// order of the last rebuild and the pair kernel classifies each atom's stored
// list V(i); a rebuild (counting sort, then the stencil walk at r_s + skin
// writing V) happens on the first call, after n or the skin changed, and
// when some atom has moved more than skin/2 since the last rebuild -- a test
// on the device whose answer the host reads (one wait per call).
int skin_prepare(rbe_ctx* ctx, int n, const double* pos, const double* q, const int32_t* type, const int32_t* mol,
                 cudaStream_t st)
{
    bool rebuild = !ctx->skin_valid || ctx->skin_n != n;
    if (!rebuild) {
        int moved = 0;
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->skin_moved, 0, sizeof(int), st));
        launch_skin_gather(ctx, n, pos, q, type, mol, st);
        CUDA_TRY(ctx, cudaMemcpyAsync(&moved, ctx->skin_moved, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(ctx, cudaStreamSynchronize(st));
        rebuild = moved != 0;
    }
    if (rebuild) {
        launch_quantize_count(ctx, n, pos, q, type, mol, st);
        launch_scan(ctx, st);
        launch_scatter_sort_gather(ctx, n, st);
        launch_skin_mark(ctx, n, st);
        launch_rbl_build(ctx, n, st);
        ctx->skin_valid = 1;
        ctx->skin_n = n;
        ctx->skin_rebuilds++;
    }
    return RBE_OK;
}

int forces_device(rbe_ctx* ctx, uint64_t step, int n, const double* pos, const double* q, const int32_t* type,
                  const int32_t* mol, double* F, cudaStream_t st)
{
    ctx->last_launches = 0;
    const bool skin = ctx->skin > 0.0;
    if (skin) {
        int rc = skin_prepare(ctx, n, pos, q, type, mol, st);
        if (rc) return rc;
    } else {
        launch_quantize_count(ctx, n, pos, q, type, mol, st);
        launch_scan(ctx, st);
        launch_scatter_sort_gather(ctx, n, st);
    }
    // the k samples and structure factors need only the sorted arrays: on an
    // auxiliary stream they run beside the pair kernel, whose last wave
    // leaves SMs idle that they can fill; joined before the finalisation.
    // With per-kernel profiling on they stay on the caller's stream: the
    // event interval of a kernel on a concurrent stream includes its wait for
    // SMs held by the pair kernel
    bool aux = RBE_OVERLAP_KSPACE != 0 && !ctx->profiling;
    if (aux && !ctx->st_aux) {
        if (cudaStreamCreateWithFlags(&ctx->st_aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return set_err(ctx, RBE_ECUDA, "cannot create the auxiliary stream");
        }
    }
    cudaStream_t sk = aux ? ctx->st_aux : st;
    if (aux) {
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, st));
        CUDA_TRY(ctx, cudaStreamWaitEvent(sk, ctx->ev_fork, 0));
    }
    launch_ksample(ctx, step, sk);
    launch_rho(ctx, n, sk);
    if (aux) CUDA_TRY(ctx, cudaEventRecord(ctx->ev_join, sk));
    if (skin) launch_rbl_stored(ctx, n, step, st);
    else launch_rbl(ctx, n, step, st);
    if (aux) CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0));
    if (ctx->n_wmol > 0) launch_bonded(ctx, n, pos, st);
    launch_finalize(ctx, n, st);
    launch_kforce(ctx, n, F, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, RBE_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return RBE_OK;
}

int copy_out(rbe_ctx* ctx, double* dst, const double* src, int count, cudaStream_t st, bool* need_sync)
{
    if (!dst) return RBE_OK;
    if (is_device_ptr(dst)) {
        CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToDevice, st));
    } else {
        CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
        *need_sync = true;
    }
    return RBE_OK;
}

int status_code(int bits)
{
    if (bits & RBE_ST_OVERLAP) return RBE_EOVERLAP;
    if (bits & RBE_ST_CAPACITY) return RBE_ECAPACITY;
    if (bits & RBE_ST_NONFINITE) return RBE_ENONFINITE;
    if (bits & RBE_ST_NONNEUTRAL) return RBE_ENONNEUTRAL;
    if (bits & RBE_ST_BADTYPE) return RBE_EINVAL;
    if (bits & RBE_ST_KSAMPLE) return RBE_ECUDA;
    if (bits & RBE_ST_STAGE) return RBE_ECUDA;
    return RBE_OK;
}

// Waits for the stream, reads the device status block into w and resets it
// (bits and needed capacities to 0, halt code to -1).
int read_status(rbe_ctx* ctx, cudaStream_t st, int w[RBE_STW_WORDS])
{
    const int init[RBE_STW_WORDS] = {0, 0, 0, -1, 0};
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    CUDA_TRY(ctx, cudaMemcpy(w, ctx->status, sizeof(int) * RBE_STW_WORDS, cudaMemcpyDeviceToHost));
    CUDA_TRY(ctx, cudaMemcpy(ctx->status, init, sizeof(init), cudaMemcpyHostToDevice));
    return RBE_OK;
}

// After a list overflow: capacities that hold the largest counts met (plus
// a margin, never smaller than before).  The next ensure() lays out shared
// memory for them, or fails with RBE_ECAPACITY if they cannot fit.
void grow_caps(rbe_ctx* ctx, const int w[RBE_STW_WORDS])
{
    int cc = w[RBE_STW_NEED_CORE] + 32, sc = w[RBE_STW_NEED_SHELL] + 32;
    cc = cc > ctx->core_cap ? cc : ctx->core_cap;
    sc = sc > ctx->shell_cap ? sc : ctx->shell_cap;
    cc = (cc + 31) / 32 * 32;
    if (sc < cc + RBE_RBL_PAIR_CARVE) sc = cc + RBE_RBL_PAIR_CARVE;     // room for the two-atom path
    ctx->user_core_cap = cc;
    if (w[RBE_STW_NEED_LIST] > 0) ctx->skin_vcap_min = w[RBE_STW_NEED_LIST] + 64;
    ctx->user_shell_cap = (sc + 31) / 32 * 32;
    ctx->last_n = -1;           // recompute caps, geometry and grids
}

}  // namespace

// ---------------------------------------------------------------------------
// profiling helpers
// ---------------------------------------------------------------------------
const char* const KERNEL_NAMES[RBE_NKERNELS] = {"quantize", "scan", "scatter", "sort", "gather", "ksample", "rho",
                                                "rhosum", "rbl", "bonded", "finalize", "kforce", "vv", "misc",
                                                "skin"};

// With profiling on, every launch is bracketed by CUDA events (timing) and an
// NVTX range named after the kernel (for timeline tools).
void prof_begin(rbe_ctx* ctx, int kid, cudaStream_t st)
{
    ctx->last_launches++;
    if (!ctx->profiling) return;
    nvtxRangePushA(KERNEL_NAMES[kid]);
    ProfState* ps = (ProfState*)ctx->prof;
    cudaEvent_t a;
    if (!ps->pool.empty()) { a = ps->pool.back(); ps->pool.pop_back(); }
    else cudaEventCreate(&a);
    cudaEventRecord(a, st);
    ps->pending_a = a;
}

void prof_end(rbe_ctx* ctx, int kid, cudaStream_t st)
{
    if (!ctx->profiling) return;
    ProfState* ps = (ProfState*)ctx->prof;
    cudaEvent_t b;
    if (!ps->pool.empty()) { b = ps->pool.back(); ps->pool.pop_back(); }
    else cudaEventCreate(&b);
    cudaEventRecord(b, st);
    ps->recs.push_back({kid, ps->pending_a, b});
    nvtxRangePop();
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int rbe_create(rbe_ctx** out, double box_L, double alpha, double r_c, double r_s, int p, int P, uint64_t seed)
{
    if (!out) return RBE_EINVAL;
    *out = nullptr;
    if (!(box_L > 0) || !(alpha > 0) || !(r_c > 0) || !(r_s > r_c) || !(r_s <= 0.5 * box_L) || p < 1 || P < 1 ||
        !isfinite(box_L) || !isfinite(alpha))
        return RBE_EINVAL;
    int n_cell = (int)floor(box_L / r_c);
    long ncells = (long)n_cell * n_cell * n_cell;
    if (n_cell < 1 || ncells > (1L << 26) || p > 512 || P > (1 << 20)) return RBE_EINVAL;
    rbe_ctx* ctx = (rbe_ctx*)calloc(1, sizeof(rbe_ctx));
    if (!ctx) return RBE_ENOMEM;
    ctx->prof = new ProfState();
    RbeConsts& c = ctx->c;
    c.L = box_L; c.alpha = alpha; c.r_c = r_c; c.r_s = r_s; c.k_e = 1.0; c.p = p; c.P = P; c.seed = seed;
    c.n_cell = n_cell;
    c.reach = (int)floor(r_s * (double)n_cell / box_L) + 1;
    c.Rc2 = radius2_fixed(r_c, box_L);
    c.Rs2 = radius2_fixed(r_s, box_L);
    c.rs_frac2 = (float)((r_s / box_L) * (r_s / box_L) * (1.0 + 1e-4));
    c.M = k_truncation(alpha, box_L);
    {
        std::vector<uint64_t> T(2 * c.M + 1);
        double H = k_thresholds(alpha, box_L, c.M, T.data());
        c.S = H * H * H - 1.0;
    }
    c.ntypes = 1;
    c.shift_lj = 0;
    ctx->eps[0] = 0.0;
    ctx->sigma[0] = 1.0;
    ctx->ncells = ncells;
    ctx->device = -1;
    ctx->last_n = -1;
    ctx->halt_step = -1;
    ctx->last_precision = -1;
    ctx->precision = RBE_FP64;
    refresh_consts(ctx);
    *out = ctx;
    return RBE_OK;
}

int rbe_set_coulomb(rbe_ctx* ctx, double k_e)
{
    if (!ctx || !isfinite(k_e)) return RBE_EINVAL;
    ctx->c.k_e = k_e;
    refresh_consts(ctx);
    return RBE_OK;
}

int rbe_set_lj(rbe_ctx* ctx, int ntypes, const double* eps, const double* sigma, int shift_energy)
{
    if (!ctx) return RBE_EINVAL;
    if (ntypes < 1 || ntypes > RBE_MAXT || !eps || !sigma)
        return set_err(ctx, RBE_EINVAL, "ntypes must be in [1, %d] with eps and sigma given", RBE_MAXT);
    for (int t = 0; t < ntypes; ++t) {
        if (!(eps[t] >= 0) || !(sigma[t] > 0)) return set_err(ctx, RBE_EINVAL, "bad LJ parameters for type %d", t);
        ctx->eps[t] = eps[t];
        ctx->sigma[t] = sigma[t];
    }
    ctx->c.ntypes = ntypes;
    ctx->c.shift_lj = shift_energy ? 1 : 0;
    ctx->lj_dirty = 1;
    return RBE_OK;
}

int rbe_set_precision(rbe_ctx* ctx, int mode)
{
    if (!ctx || (mode != RBE_FP64 && mode != RBE_MIXED)) return RBE_EINVAL;
    ctx->precision = mode;
    return RBE_OK;
}

int rbe_set_water_bonds(rbe_ctx* ctx, int n_mol, double k_b, double r0, double k_theta, double theta0)
{
    if (!ctx || n_mol < 0) return RBE_EINVAL;
    ctx->n_wmol = n_mol;
    ctx->kb = k_b; ctx->r0 = r0; ctx->kth = k_theta; ctx->th0 = theta0;
    return RBE_OK;
}

int rbe_set_capacity(rbe_ctx* ctx, int core_cap, int shell_cap)
{
    if (!ctx || core_cap < 0 || shell_cap < 0) return RBE_EINVAL;
    ctx->user_core_cap = core_cap;
    ctx->user_shell_cap = shell_cap;
    ctx->last_n = -1;
    return RBE_OK;
}

int rbe_set_shell_sampling(rbe_ctx* ctx, int mode)
{
    if (!ctx || (mode != RBE_SHELL_FLOYD && mode != RBE_SHELL_REPLACE)) return RBE_EINVAL;
    ctx->c.shell_mode = mode;
    return RBE_OK;
}

int rbe_set_lj_cutoff(rbe_ctx* ctx, double factor)
{
    if (!ctx || !(factor >= 0.0) || !isfinite(factor)) return RBE_EINVAL;
    ctx->lj_rc_factor = factor;
    ctx->lj_dirty = 1;
    return RBE_OK;
}

int rbe_set_kpool(rbe_ctx* ctx, int size, int burn_in)
{
    if (!ctx || size < 0 || burn_in < 0) return RBE_EINVAL;
    ctx->c.kpool = size;
    ctx->kpool_burn = burn_in;
    ctx->kpool_dirty = 1;
    return RBE_OK;
}

int rbe_set_langevin(rbe_ctx* ctx, double kT, double tau)
{
    if (!ctx || !isfinite(kT) || !isfinite(tau) || kT < 0.0) return RBE_EINVAL;
    ctx->lang_kT = kT;
    ctx->lang_tau = tau > 0.0 ? tau : 0.0;
    ctx->lang_valid = 0;
    return RBE_OK;
}

int rbe_get_langevin_force(rbe_ctx* ctx, int n, double* FL, uint64_t* step)
{
    if (!ctx || !FL || !step || n < 1) return RBE_EINVAL;
    if (!ctx->lang_valid || ctx->lang_n != n || !ctx->F_lang)
        return set_err(ctx, RBE_EINVAL, "no Langevin force for %d atoms is held", n);
    CUDA_TRY(ctx, cudaMemcpy(FL, ctx->F_lang, sizeof(double) * 3 * (size_t)n, cudaMemcpyDefault));
    *step = ctx->lang_step;
    return RBE_OK;
}

int rbe_set_langevin_force(rbe_ctx* ctx, int n, const double* FL, uint64_t step)
{
    if (!ctx || !FL || n < 1) return RBE_EINVAL;
    int rc = ensure(ctx, n);
    if (rc) return rc;
    if ((rc = ctx_grow_lang(ctx, n))) return rc;
    CUDA_TRY(ctx, cudaMemcpy(ctx->F_lang, FL, sizeof(double) * 3 * (size_t)n, cudaMemcpyDefault));
    ctx->lang_step = step;
    ctx->lang_valid = 1;
    ctx->lang_n = n;
    return RBE_OK;
}

int rbe_set_verlet_skin(rbe_ctx* ctx, double skin)
{
    if (!ctx) return RBE_EINVAL;
    if (!(skin >= 0.0) || (skin > 0.0 && ctx->c.r_s + skin > 0.5 * ctx->c.L))
        return set_err(ctx, RBE_EINVAL, "skin must be >= 0 with r_s + skin <= L/2");
    ctx->skin_valid = 0;        // the next call rebuilds
    if (skin != ctx->skin) {
        ctx->skin = skin;
        ctx->skin_vcap_min = 0;
        ctx->last_n = -1;       // recompute the geometry (and the list build's) at the next call
    }
    return RBE_OK;
}

int rbe_set_rbl_tiling(rbe_ctx* ctx, int atoms_per_unit, int units_per_slot)
{
    if (!ctx || atoms_per_unit < 0 || units_per_slot < 0 || atoms_per_unit > 4096) return RBE_EINVAL;
    ctx->tune_apu = atoms_per_unit;
    ctx->tune_ups = units_per_slot;
    ctx->last_n = -1;
    return RBE_OK;
}

int rbe_set_debug(rbe_ctx* ctx, int on, int cap_core)
{
    if (!ctx || cap_core < 0) return RBE_EINVAL;
    ctx->debug = on ? 1 : 0;
    ctx->dbg_cap_core = cap_core;
    ctx->dbg_n_cap = 0;
    return RBE_OK;
}

int rbe_set_profiling(rbe_ctx* ctx, int on)
{
    if (!ctx) return RBE_EINVAL;
    ctx->profiling = on ? 1 : 0;
    return RBE_OK;
}

int rbe_forces(rbe_ctx* ctx, uint64_t step, int n, const double* pos, const double* q, const int32_t* type,
               const int32_t* mol, double* F, double* energy, double* virial, void* cuda_stream)
{
    if (!ctx) return RBE_EINVAL;
    if (n < 1 || !pos || !q || !F) return set_err(ctx, RBE_EINVAL, "n >= 1 and pos, q, F are required");
    if (ctx->n_wmol > 0 && 3 * ctx->n_wmol > n)
        return set_err(ctx, RBE_EINVAL, "water bonds cover %d atoms but n = %d", 3 * ctx->n_wmol, n);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = ensure(ctx, n);
    if (rc) return rc;
    bool dev_in = is_device_ptr(pos);
    if (dev_in != is_device_ptr(q) || dev_in != is_device_ptr(F) || (type && dev_in != is_device_ptr(type)) ||
        (mol && dev_in != is_device_ptr(mol)))
        return set_err(ctx, RBE_EINVAL, "pos, q, type, mol and F must all be device or all host pointers");
    bool need_sync = false;
    if (dev_in) {
        rc = forces_device(ctx, step, n, pos, q, type, mol, F, st);
    } else {
        if (n > ctx->h_cap) {
            // each dev_alloc frees the old buffer first: a failure part way
            // leaves the set incomplete, so the capacity is zero until all
            // five succeed
            ctx->h_cap = 0;
            if ((rc = dev_alloc(ctx, &ctx->h_pos, 3 * (size_t)n))) return rc;
            if ((rc = dev_alloc(ctx, &ctx->h_q, n))) return rc;
            if ((rc = dev_alloc(ctx, &ctx->h_type, n))) return rc;
            if ((rc = dev_alloc(ctx, &ctx->h_mol, n))) return rc;
            if ((rc = dev_alloc(ctx, &ctx->h_F, 3 * (size_t)n))) return rc;
            ctx->h_cap = n;
        }
        // inputs in pinned host memory that the device can address are read in
        // place: the quantisation reads them once, in order, and everything
        // after it reads its device copies (the Verlet-skin path reads the
        // positions in sorted order and takes the copies)
        const double* vpos = (const double*)pinned_device_view(pos);
        const double* vq = (const double*)pinned_device_view(q);
        const int32_t* vtype = type ? (const int32_t*)pinned_device_view(type) : nullptr;
        const int32_t* vmol = mol ? (const int32_t*)pinned_device_view(mol) : nullptr;
        if (ctx->skin == 0.0 && vpos && vq && (!type || vtype) && (!mol || vmol)) {
            rc = forces_device(ctx, step, n, vpos, vq, vtype, vmol, ctx->h_F, st);
        } else {
            CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
            CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_q, q, sizeof(double) * n, cudaMemcpyHostToDevice, st));
            if (type) CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_type, type, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
            if (mol) CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_mol, mol, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
            rc = forces_device(ctx, step, n, ctx->h_pos, ctx->h_q, type ? ctx->h_type : nullptr,
                               mol ? ctx->h_mol : nullptr, ctx->h_F, st);
        }
        if (rc) return rc;
        CUDA_TRY(ctx, cudaMemcpyAsync(F, ctx->h_F, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
        need_sync = true;
    }
    if (rc) return rc;
    if ((rc = copy_out(ctx, energy, ctx->totals, RBE_NE, st, &need_sync))) return rc;
    if ((rc = copy_out(ctx, virial, ctx->totals + 6, RBE_NW, st, &need_sync))) return rc;
    if (need_sync) {
        // the call waits anyway: a list overflow is retried once with
        // capacities that hold the counts met (other errors stay latched for
        // rbe_sync_status)
        int w[RBE_STW_WORDS];
        if ((rc = read_status(ctx, st, w))) return rc;
        if (w[0] == RBE_ST_CAPACITY && !ctx->retrying) {
            grow_caps(ctx, w);
            ctx->retrying = 1;
            rc = rbe_forces(ctx, step, n, pos, q, type, mol, F, energy, virial, cuda_stream);
            ctx->retrying = 0;
            return rc;
        }
        if (w[0]) CUDA_TRY(ctx, cudaMemcpy(ctx->status, w, sizeof(int), cudaMemcpyHostToDevice));
    }
    return RBE_OK;
}

int rbe_step(rbe_ctx* ctx, uint64_t step0, int nsteps, double dt, double accel, int n, double* pos, double* vel,
             const double* mass, const double* q, const int32_t* type, const int32_t* mol, double* F,
             double* energy_trace, void* cuda_stream)
{
    if (!ctx) return RBE_EINVAL;
    if (nsteps < 0 || n < 1 || !pos || !vel || !mass || !q || !F || !(dt > 0) || !(accel > 0))
        return set_err(ctx, RBE_EINVAL, "bad rbe_step arguments");
    if (!is_device_ptr(pos) || !is_device_ptr(vel) || !is_device_ptr(mass) || !is_device_ptr(F))
        return set_err(ctx, RBE_EINVAL, "rbe_step takes device pointers");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = ensure(ctx, n);
    if (rc) return rc;
    // Langevin thermostat: F^L from the entry velocities at step0, then after
    // every force evaluation from the half-kicked velocities
    // (a call that starts where the context's previous run ended reuses that
    // run's last F^L, so a run split into calls equals one call bit for bit)
    const bool lang = ctx->lang_tau > 0.0;
    if (lang) {
        if ((rc = ctx_grow_lang(ctx, n))) return rc;
        if (!(ctx->lang_valid && ctx->lang_step == step0 && ctx->lang_n == n))
            launch_langevin(ctx, n, vel, mass, step0, dt, accel, st);
    }
    const double* FL = lang ? ctx->F_lang : nullptr;
    // the second half of step k: forces at step0 + k + 1, thermostat, kick
    auto finish_step = [&](int k) -> int {
        int r = forces_device(ctx, step0 + (uint64_t)k + 1, n, pos, q, type, mol, F, st);
        if (r) return r;
        if (lang) launch_langevin(ctx, n, vel, mass, step0 + (uint64_t)k + 1, dt, accel, st);
        launch_vv_kick_drift(ctx, n, pos, vel, mass, F, FL, dt, accel, 0, 2 * k + 1, st);
        if (energy_trace) launch_ke_trace(ctx, n, vel, mass, accel, energy_trace + 2 * (size_t)k, st);
        return RBE_OK;
    };
    auto run = [&](int k0) -> int {
        for (int k = k0; k < nsteps; ++k) {
            launch_vv_kick_drift(ctx, n, pos, vel, mass, F, FL, dt, accel, 1, 2 * k, st);
            int r = finish_step(k);
            if (r) return r;
        }
        return RBE_OK;
    };
    ctx->halt_step = -1;
    if ((rc = run(0))) return rc;
    // A latched error stops the integration on the device (the kicks leave
    // positions and velocities as they are).  A list overflow in the force
    // evaluation of step k is retried once: capacities grown to the counts
    // met, that evaluation and the second half kick redone, the remaining
    // steps run.
    int w[RBE_STW_WORDS];
    if ((rc = read_status(ctx, st, w))) return rc;
    if (w[0] == RBE_ST_CAPACITY && w[RBE_STW_HALT] >= 0 && (w[RBE_STW_HALT] & 1)) {
        const int k = w[RBE_STW_HALT] >> 1;
        grow_caps(ctx, w);
        if ((rc = ensure(ctx, n))) return rc;
        if ((rc = finish_step(k))) return rc;
        if ((rc = run(k + 1))) return rc;
        if ((rc = read_status(ctx, st, w))) return rc;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, RBE_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    if (w[0]) {
        // stopped: the state is the one after the launch before the stop; the
        // status stays latched for rbe_sync_status
        const int h = w[RBE_STW_HALT];
        ctx->halt_step = h < 0 ? -1 : (long long)(step0 + (uint64_t)(h >> 1) + (uint64_t)(h & 1));
        ctx->lang_valid = 0;
        CUDA_TRY(ctx, cudaMemcpy(ctx->status, w, sizeof(int), cudaMemcpyHostToDevice));
        const int code = status_code(w[0]);
        return set_err(ctx, code, "integration stopped at the force evaluation of step %lld (status bits 0x%x)",
                       ctx->halt_step, w[0]);
    }
    if (lang) {
        ctx->lang_step = step0 + (uint64_t)nsteps;
        ctx->lang_valid = 1;
        ctx->lang_n = n;
    }
    return RBE_OK;
}

int rbe_adjoint(rbe_ctx* ctx, uint64_t step, int n, const double* pos, const double* q, const int32_t* type,
                const int32_t* mol, const double* gF, double* dEdq, double* dLdq, double* dEdeps, double* dEdsig,
                double* dLdeps, double* dLdsig, void* cuda_stream)
{
    if (!ctx) return RBE_EINVAL;
    if (ctx->skin > 0.0)
        return set_err(ctx, RBE_EINVAL, "rbe_adjoint differentiates the stencil lists: turn the Verlet skin off");
    if (n < 1 || !pos || !q) return set_err(ctx, RBE_EINVAL, "n >= 1 and pos, q are required");
    if (!is_device_ptr(pos) || !is_device_ptr(q) || (type && !is_device_ptr(type)) || (mol && !is_device_ptr(mol)) ||
        (gF && !is_device_ptr(gF)) || (dEdq && !is_device_ptr(dEdq)) || (dLdq && !is_device_ptr(dLdq)))
        return set_err(ctx, RBE_EINVAL, "rbe_adjoint takes device pointers for per-atom arrays");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = ensure(ctx, n);
    if (rc) return rc;
    const int nt2 = ctx->c.ntypes * ctx->c.ntypes;
    if ((rc = grow(ctx, &ctx->vs, &ctx->cap_atoms[18], 3 * (size_t)n))) return rc;
    if ((rc = grow(ctx, &ctx->gq_own, &ctx->cap_atoms[19], 2 * (size_t)n))) return rc;
    if ((rc = grow(ctx, &ctx->gq_tr, &ctx->cap_adj[0], 2 * (size_t)n))) return rc;
    if ((rc = grow(ctx, &ctx->part_lj, &ctx->cap_adj[1], (size_t)ctx->grid_rbl * 4 * nt2))) return rc;
    if ((rc = grow(ctx, &ctx->part_v, &ctx->cap_adj[2], (size_t)ctx->grid_q * 3))) return rc;
    if ((rc = grow(ctx, &ctx->tau_part, &ctx->cap_adj[3], (size_t)ctx->grid_rho * ctx->c.P))) return rc;
    if ((rc = grow(ctx, &ctx->tau, &ctx->cap_adj[4], (size_t)ctx->c.P))) return rc;
    ctx->last_launches = 0;
    // the forward set-up of the same step: identical lists, batches, k samples
    launch_quantize_count(ctx, n, pos, q, type, mol, st);
    launch_scan(ctx, st);
    launch_scatter_sort_gather(ctx, n, st);
    launch_ksample(ctx, step, st);
    launch_rho(ctx, n, st);
    launch_adj_prep(ctx, n, gF, st);
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->gq_tr, 0, sizeof(double) * 2 * (size_t)n, st));
    launch_rbl(ctx, n, step, st, true);
    launch_adj_final(ctx, n, dEdq, dLdq, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, RBE_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    // LJ pair-parameter partials: fixed-order sum, then the Lorentz-Berthelot
    // chain rule to per-type parameters (eps_ab = sqrt(eps_a eps_b),
    // sigma_ab = (sigma_a + sigma_b)/2)
    std::vector<double> part((size_t)ctx->grid_rbl * 4 * nt2);
    CUDA_TRY(ctx, cudaMemcpyAsync(part.data(), ctx->part_lj, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    const int T = ctx->c.ntypes;
    std::vector<double> g(4 * (size_t)nt2, 0.0);
    for (int b = 0; b < ctx->grid_rbl; ++b)
        for (int k = 0; k < 4 * nt2; ++k) g[k] += part[(size_t)b * 4 * nt2 + k];
    double* outs[4] = {dEdeps, dEdsig, dLdeps, dLdsig};
    for (int o = 0; o < 4; ++o) {
        if (!outs[o]) continue;
        const double* go = g.data() + (size_t)o * nt2;
        for (int a2 = 0; a2 < T; ++a2) {
            double acc = 0.0;
            for (int b2 = 0; b2 < T; ++b2) {
                const double sym = a2 == b2 ? go[a2 * T + a2] : go[a2 * T + b2] + go[b2 * T + a2];
                double dpar;
                if (o == 0 || o == 2) {   // eps
                    if (a2 == b2) dpar = 1.0;
                    else if (ctx->eps[b2] == 0.0) dpar = 0.0;
                    else if (ctx->eps[a2] == 0.0) dpar = HUGE_VAL;
                    else dpar = ctx->eps[b2] / (2.0 * sqrt(ctx->eps[a2] * ctx->eps[b2]));
                } else {                  // sigma
                    dpar = a2 == b2 ? 1.0 : 0.5;
                }
                if (sym != 0.0) acc += sym * dpar;
            }
            outs[o][a2] = acc;
        }
    }
    return RBE_OK;
}

int rbe_sync_status(rbe_ctx* ctx, void* cuda_stream)
{
    if (!ctx) return RBE_EINVAL;
    if (!ctx->status) return RBE_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int w[RBE_STW_WORDS];
    int rc = read_status(ctx, st, w);
    if (rc) return rc;
    // a list overflow sizes the next call's capacities to the counts met
    if (w[0] & RBE_ST_CAPACITY) grow_caps(ctx, w);
    int code = status_code(w[0]);
    if (code) set_err(ctx, code, "device status bits 0x%x", w[0]);
    return code;
}

int rbe_get_lists(rbe_ctx* ctx, int n, int32_t* n_core, int32_t* n_shell, int32_t* core, int32_t* batch,
                  void* cuda_stream)
{
    if (!ctx) return RBE_EINVAL;
    if (!ctx->dbg_ncore || n > ctx->dbg_n_cap) return set_err(ctx, RBE_EINVAL, "no recorded lists for n = %d", n);
    CUDA_TRY(ctx, cudaStreamSynchronize((cudaStream_t)cuda_stream));
    if (n_core) CUDA_TRY(ctx, cudaMemcpy(n_core, ctx->dbg_ncore, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (n_shell) CUDA_TRY(ctx, cudaMemcpy(n_shell, ctx->dbg_nshell, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (core && ctx->dbg_cap_core > 0)
        CUDA_TRY(ctx, cudaMemcpy(core, ctx->dbg_core, sizeof(int) * (size_t)n * ctx->dbg_cap_core, cudaMemcpyDeviceToHost));
    if (batch) CUDA_TRY(ctx, cudaMemcpy(batch, ctx->dbg_batch, sizeof(int) * (size_t)n * ctx->c.p, cudaMemcpyDeviceToHost));
    return RBE_OK;
}

int rbe_get_kspace(rbe_ctx* ctx, int32_t* m, double* rho, void* cuda_stream)
{
    if (!ctx) return RBE_EINVAL;
    if (!ctx->km) return set_err(ctx, RBE_EINVAL, "no step has run");
    CUDA_TRY(ctx, cudaStreamSynchronize((cudaStream_t)cuda_stream));
    if (m) {
        std::vector<int4> h(ctx->c.P);
        CUDA_TRY(ctx, cudaMemcpy(h.data(), ctx->km, sizeof(int4) * ctx->c.P, cudaMemcpyDeviceToHost));
        for (int l = 0; l < ctx->c.P; ++l) { m[3 * l] = h[l].x; m[3 * l + 1] = h[l].y; m[3 * l + 2] = h[l].z; }
    }
    if (rho) CUDA_TRY(ctx, cudaMemcpy(rho, ctx->rho, sizeof(double2) * ctx->c.P, cudaMemcpyDeviceToHost));
    return RBE_OK;
}

int rbe_get_info(rbe_ctx* ctx, double* out, int nout)
{
    if (!ctx || !out) return RBE_EINVAL;
    int dbg[2] = {-1, -1};
    if (nout > 7 && ctx->debug && ctx->dbg_unstaged)
        CUDA_TRY(ctx, cudaMemcpy(dbg, ctx->dbg_unstaged, sizeof(dbg), cudaMemcpyDeviceToHost));
    double v[12] = {(double)ctx->c.n_cell, (double)ctx->c.reach, (double)ctx->c.M, ctx->c.S, (double)ctx->core_cap,
                    (double)ctx->shell_cap, (double)ctx->last_launches, (double)dbg[0], (double)dbg[1],
                    (double)ctx->halt_step, (double)ctx->skin_rebuilds, (double)ctx->skin_vcap};
    for (int k = 0; k < nout && k < 12; ++k) out[k] = v[k];
    return RBE_OK;
}

int rbe_get_profile(rbe_ctx* ctx, double* ms, int64_t* launches, int reset, void* cuda_stream)
{
    if (!ctx) return RBE_EINVAL;
    CUDA_TRY(ctx, cudaStreamSynchronize((cudaStream_t)cuda_stream));
    ProfState* ps = (ProfState*)ctx->prof;
    for (auto& r : ps->recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ctx->prof_ms[r.kid] += t;
            ctx->prof_n[r.kid] += 1;
        }
        ps->pool.push_back(r.a);
        ps->pool.push_back(r.b);
    }
    ps->recs.clear();
    for (int k = 0; k < RBE_NKERNELS; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->prof_n[k];
    }
    if (reset)
        for (int k = 0; k < RBE_NKERNELS; ++k) { ctx->prof_ms[k] = 0.0; ctx->prof_n[k] = 0; }
    return RBE_OK;
}

const char* rbe_last_error(const rbe_ctx* ctx) { return ctx ? ctx->err : "null context"; }

void rbe_destroy(rbe_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->device >= 0) {
        ProfState* ps = (ProfState*)ctx->prof;
        for (auto& r : ps->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : ps->pool) cudaEventDestroy(e);
        free_dev(ctx);
        if (ctx->st_aux) {
            cudaEventDestroy(ctx->ev_fork);
            cudaEventDestroy(ctx->ev_join);
            cudaStreamDestroy(ctx->st_aux);
        }
    }
    delete (ProfState*)ctx->prof;
    free(ctx);
}

}  // extern "C"
