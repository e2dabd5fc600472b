/*
 * rbe_oracle.c -- plain FP64 CPU oracle for the improved random batch Ewald
 * (IRBE = RBL real space + RBE Fourier space) force step of
 * Liang, Xu & Zhao, "Improved random batch Ewald method in molecular dynamics
 * simulations" (arXiv 2204.13595).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, the smoke check and the CPU-baseline leg of bench.py load it.
 * It shares no code with the CUDA library; the two agree only through the
 * definitions below, each of which cites the passage of the paper it follows.
 *
 * Everything is IEEE double, compiled with -ffp-contract=off, written as the
 * plain definition (no blocking, fusion or reordering beyond what the
 * definition states).  OpenMP is used only over independent atoms; every
 * reduction over atoms is a sequential loop in atom order.
 *
 * Readings of the paper taken here (the paper is silent on these):
 *  R1  The paper's core radius r_eta is called r_c here and its outer cutoff
 *      r_c is called r_s.  Core C(i) = {j != i : r_ij <= r_c}, shell
 *      S(i) = {j : r_c < r_ij <= r_s} (Sec. 2.3, definition of C(i), S(i)).
 *  R2  Set membership is decided on 32-bit fixed-point fractional coordinates
 *      s = floor(frac(x/L) * 2^32): the squared distance is the exact integer
 *      sum of squared wrapped differences, compared with floor((r*2^32/L)^2).
 *      This makes list membership reproducible bit for bit.
 *  R3  The shell batch B(i) is drawn uniformly without replacement by Floyd's
 *      algorithm (Bentley & Floyd, CACM 1987) over ordinals [0, N_S); ordinals
 *      index S(i) in canonical order: ascending (cell index, fixed-point x
 *      code s_x, atom id) on the grid of n_cell = floor(L/r_c) cells per axis
 *      (Sec. 2.3 uses cells of edge r_eta).  If N_S <= p the batch is all of S(i) with weight 1
 *      (Algorithm 1, shell selection step).
 *  R4  The k sampler draws each axis independently from the discrete Gaussian
 *      w_m = exp(-pi^2 m^2 / (alpha L^2)) by exact inverse CDF on 64-bit
 *      thresholds, and redraws (0,0,0); this is exactly P_k of Eq. (2.8)
 *      (the paper uses rounding plus Metropolis-Hastings for the same law).
 *      Fresh iid samples are drawn every step.
 *  R5  Random numbers: Philox4x64-10 (Salmon et al., SC'11), key (seed, 0),
 *      counter (a, b, step, stream).  Shell slot k of atom i uses word k%4 of
 *      the block at counter (i, k/4, step, 1).  k sample l, attempt t uses
 *      words 0..2 of the block at counter (l, t, step, 2).
 *  R6  Pair f_ij is Eq. (2.10) with a Coulomb prefactor k_e; LJ uses
 *      Lorentz-Berthelot mixing; force truncated at r_s (unshifted), energy
 *      optionally shifted to zero at r_s.
 *  R7  Same-molecule (excluded) pairs keep their membership in C(i)/S(i) but
 *      their pair term is the Ewald exclusion correction
 *      -k_e q_i q_j erf(sqrt(alpha) r)/r instead of erfc + LJ.
 *  R13 Variants (Algorithm 1 and Sec. 2.3 leave these open): shell_mode 1
 *      draws the p slots of B(i) independently and uniformly with
 *      replacement (same words, ordinal floor(u N_S / 2^64)), weight N_S/p;
 *      lj_rc_factor f > 0 truncates the LJ term of pair (a, b) at
 *      min(f sigma_ab, r_s), shifted there when shift_lj is set (f = 2^(1/6)
 *      with the shift is the WCA soft sphere of the paper's electrolytes,
 *      Sec. 3.1); kpool K > 0 replaces the fresh draws of R4 by the pool of
 *      Algorithm 1: K samples of a Metropolis-Hastings chain per axis
 *      (proposal round(x), x ~ N(0, alpha L^2 / (2 pi^2)), Sec. 2.2), and
 *      sample l of a step is pool entry floor(u K / 2^64), u word 0 of the
 *      block at counter (l, 0, step, 5).
 *  R14 Langevin thermostat (Sec. 3.1 runs the electrolytes with a Langevin
 *      thermostat of relaxation time tau inside velocity Verlet; the form is
 *      not given): with force-to-acceleration factor accel, each force
 *      evaluation at step s adds F^L_i = -(m_i / (accel tau)) v_i
 *      + sqrt(24 m_i kT / (accel tau dt)) (u - 1/2) per component, v_i the
 *      velocity at that moment (after the first half kick), u = (w >> 11)
 *      2^-53 from word a of the Philox block at counter (i, 0, s, 3): a
 *      uniform random force of the variance 2 m kT / (accel tau dt) of the
 *      Euler-Maruyama step; the first half kick of the next step uses it too.
 *  R15 Verlet skin (Sec. 2.3 remarks that cells slightly larger than r_eta
 *      spare rebuilding the lists every step; the scheme is not given): with
 *      skin d > 0, a stored list V(i) = {j != i : r_ij <= r_s + d} is built
 *      from the positions of a rebuild step t_b, by the exact rule of R2 with
 *      floor(((r_s + d) 2^32/L)^2), in the canonical order of R3 at t_b.  At
 *      a later step the sets C(i), S(i) are the members of V(i) classified by
 *      R2 at the current positions, kept in the order of V(i); the ordinals
 *      of R3 index S(i) in that order.  A rebuild is due when some atom's
 *      fixed-point displacement since t_b, sum_a (int32)(s_a - s_a(t_b))^2,
 *      exceeds floor((d/2 2^32/L)^2): below it every pair within r_s now was
 *      within r_s + d at t_b (triangle inequality), so C(i) and S(i) equal
 *      those of the stencil at every step.
 *  R8  Energy estimator: E_real = 1/2 sum_i [sum_C u_ij + w_i sum_B u_ij];
 *      E_k = (S/P) sum_l (2 pi k_e / (V k_l^2)) |rho_l|^2;
 *      E_self = -k_e sqrt(alpha/pi) sum q^2  (Eq. (2.3) terms, reweighted).
 *      Virial W_ab = -1/2 sum_i sum_j w_ij (r_ij)_a (f_ij)_b (r_ij = r_j - r_i)
 *      plus the reweighted reciprocal-space Ewald virial.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXT 16
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Parameters                                                               */
/* ------------------------------------------------------------------------ */
typedef struct orc_params {
    double L;        /* cubic box edge (Sec. 2.1)                         */
    double alpha;    /* Ewald splitting parameter, erfc(sqrt(alpha) r)    */
    double r_c;      /* core radius (paper: r_eta)                        */
    double r_s;      /* outer cutoff (paper: r_c)                         */
    double k_e;      /* Coulomb prefactor                                 */
    int p;           /* shell batch size (paper: p tilde)                 */
    int P;           /* Fourier batch size (paper: p)                     */
    uint64_t seed;
    int ntypes;
    int shift_lj;    /* 1: LJ energy shifted to zero at r_s               */
    double eps[ORC_MAXT];    /* per-type LJ epsilon                       */
    double sigma[ORC_MAXT];  /* per-type LJ sigma                         */
    int shell_mode;          /* R13: 0 without replacement, 1 with         */
    double lj_rc_factor;     /* R13: 0 LJ to r_s, f > 0 cut at f sigma_ab  */
    int kpool;               /* R13: 0 fresh draws, K > 0 MH pool of K     */
    int kpool_burn;          /* R13: burn-in iterations of the MH chains   */
    double lang_kT;          /* R14: thermostat kT (energy units)         */
    double lang_tau;         /* R14: relaxation time; <= 0 thermostat off */
    double skin;             /* R15: Verlet skin d (0: lists every step)  */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3 / Table 2)       */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(prod >> 64);
    *lo = (uint64_t)prod;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void rng_block(uint64_t seed, uint64_t a, uint64_t b, uint64_t step,
                      uint64_t stream, uint64_t out[4])
{
    uint64_t ctr[4] = {a, b, step, stream};
    uint64_t key[2] = {seed, 0};
    orc_philox4x64_10(ctr, key, out);
}

/* floor(u * n / 2^64): a uniform integer in [0, n) from a 64-bit word. */
static uint64_t uniform_below(uint64_t u, uint64_t n)
{
    uint64_t hi, lo;
    mulhilo64(u, n, &hi, &lo);
    return hi;
}

/* Compensated (Neumaier) running sum: the sums over all atoms below are
 * evaluated to within a few ulp of the exact sum whatever N is, where plain
 * recursion's error bound grows as (N-1) u. */
typedef struct { double s, c; } ksum;
static void ksum_add(ksum* k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}
static double ksum_get(const ksum* k) { return k->s + k->c; }

/* ------------------------------------------------------------------------ */
/* Fixed-point coordinates and cells (readings R2, R3)                      */
/* ------------------------------------------------------------------------ */
/* Fractional coordinate of x in [0,1) and its 32-bit fixed-point code. */
static uint32_t fixed_point(double x, double invL)
{
    double t = x * invL;
    double f = t - floor(t);
    if (f >= 1.0) f = 0.0;
    return (uint32_t)(uint64_t)(f * 4294967296.0);
}

/* floor((r * 2^32 / L)^2): squared radius in fixed-point units. */
uint64_t orc_radius2_fixed(double r, double L)
{
    double invL = 1.0 / L;
    double a = (r * invL) * 4294967296.0;
    return (uint64_t)(a * a);
}

int orc_n_cell(double L, double r_c)
{
    return (int)floor(L / r_c);
}

static uint32_t cell_of(uint32_t s, int n_cell)
{
    return (uint32_t)(((uint64_t)s * (uint64_t)n_cell) >> 32);
}

static uint64_t dist2_fixed(const uint32_t* si, const uint32_t* sj)
{
    uint64_t d2 = 0;
    for (int a = 0; a < 3; ++a) {
        int32_t d = (int32_t)(sj[a] - si[a]);
        d2 += (uint64_t)((int64_t)d * (int64_t)d);
    }
    return d2;
}

/* Quantise all atoms: s[3N] fixed-point codes, cell[N] linear canonical
 * cell on the grid of n_cell = floor(L / r_c) cells per axis. */
void orc_quantize(int n, const double* pos, double L, double r_c, uint32_t* s, int32_t* cell)
{
    double invL = 1.0 / L;
    int nc = orc_n_cell(L, r_c);
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) s[3 * i + a] = fixed_point(pos[3 * i + a], invL);
        uint32_t cx = cell_of(s[3 * i + 0], nc), cy = cell_of(s[3 * i + 1], nc), cz = cell_of(s[3 * i + 2], nc);
        cell[i] = (int32_t)(cx + (uint32_t)nc * (cy + (uint32_t)nc * cz));
    }
}

/* ------------------------------------------------------------------------ */
/* k sampler (Eqs. (2.6)-(2.8), reading R4)                                 */
/* ------------------------------------------------------------------------ */
/* Truncation: |m| <= M with exp(-pi^2 M^2/(alpha L^2)) below 2^-64. */
int orc_kmax(double alpha, double L)
{
    double aL2 = alpha * L * L;
    return (int)ceil(sqrt(aL2 * 64.0 * log(2.0)) / ORC_PI);
}

/* H = sum_{|m|<=M} exp(-pi^2 m^2/(alpha L^2)) summed from m=-M upward, and
 * the thresholds T[m+M] = floor(2^64 * CDF(m)) for m = -M..M (saturating).
 * Returns H.  T must hold 2M+1 entries. */
double orc_k_table(double alpha, double L, int M, uint64_t* T)
{
    double aL2 = alpha * L * L;
    double c = ORC_PI * ORC_PI / aL2;
    double H = 0.0;
    for (int m = -M; m <= M; ++m) H += exp(-c * (double)m * (double)m);
    double acc = 0.0;
    for (int m = -M; m <= M; ++m) {
        acc += exp(-c * (double)m * (double)m);
        double cdf = acc / H;
        double v = cdf * 18446744073709551616.0;
        T[m + M] = (v >= 18446744073709551616.0) ? UINT64_MAX : (uint64_t)v;
    }
    return H;
}

/* Smallest m in [-M, M] with u < T[m+M] (m = M if none). */
static int inv_cdf(uint64_t u, const uint64_t* T, int M)
{
    for (int m = -M; m < M; ++m)
        if (u < T[m + M]) return m;
    return M;
}

/* Draw P wave vectors m_l (int[3P]) for a step; returns attempts used max. */
int orc_sample_k(uint64_t seed, uint64_t step, int P, double alpha, double L, int32_t* m_out)
{
    int M = orc_kmax(alpha, L);
    uint64_t* T = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
    orc_k_table(alpha, L, M, T);
    int worst = 0;
    for (int l = 0; l < P; ++l) {
        for (uint64_t t = 0; t < 1024; ++t) {
            uint64_t w[4];
            rng_block(seed, (uint64_t)l, t, step, 2, w);
            int mx = inv_cdf(w[0], T, M), my = inv_cdf(w[1], T, M), mz = inv_cdf(w[2], T, M);
            if (mx == 0 && my == 0 && mz == 0) continue;
            m_out[3 * l + 0] = mx; m_out[3 * l + 1] = my; m_out[3 * l + 2] = mz;
            if ((int)t > worst) worst = (int)t;
            break;
        }
    }
    free(T);
    return worst;
}

/* Metropolis-Hastings pool of k samples (R13; Algorithm 1, pool step; Sec. 2.2).
 * Per axis, target w_m = exp(-pi^2 m^2 / (alpha L^2)) and proposal
 * q_m = P(round(X) = m), X ~ N(0, s^2), s^2 = alpha L^2 / (2 pi^2), both on
 * |m| <= M (the truncation of R4) and normalised there.  Proposals are drawn
 * by inverse CDF on 64-bit thresholds of q (as R4 draws w); the move from m
 * to m* is accepted when u < (w_m* q_m) / (w_m q_m*), u = (word >> 11) 2^-53.
 * Iteration t of axis a uses the block at counter (t, a, 0, 4): word 0 the
 * proposal, word 1 the acceptance.  The chains start at 0; after `burn`
 * iterations every iteration emits (m_x, m_y, m_z) unless it is (0,0,0),
 * until K samples are collected. */
void orc_mh_tables(double alpha, double L, int M, double* w, double* q, uint64_t* Tq)
{
    double aL2 = alpha * L * L;
    double c = ORC_PI * ORC_PI / aL2;
    double s = sqrt(aL2 / (2.0 * ORC_PI * ORC_PI));
    double sq2 = s * sqrt(2.0);
    double Q = 0.0;
    for (int m = -M; m <= M; ++m) {
        w[m + M] = exp(-c * (double)m * (double)m);
        /* P(m - 1/2 <= X < m + 1/2) through complementary error functions of |m| */
        double am = fabs((double)m);
        double lo = (am - 0.5) / sq2, hi = (am + 0.5) / sq2;
        double qm = (m == 0) ? erf(0.5 / sq2) : 0.5 * (erfc(lo) - erfc(hi));
        q[m + M] = qm;
        Q += qm;
    }
    double acc = 0.0;
    for (int m = -M; m <= M; ++m) {
        acc += q[m + M];
        double v = (acc / Q) * 18446744073709551616.0;
        Tq[m + M] = (v >= 18446744073709551616.0) ? UINT64_MAX : (uint64_t)v;
    }
}

/* Fills pool[3K]; returns the accepted fraction over all axes and iterations. */
double orc_kpool(uint64_t seed, double alpha, double L, int K, int burn, int32_t* pool)
{
    int M = orc_kmax(alpha, L);
    double* w = (double*)malloc(sizeof(double) * (size_t)(2 * M + 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(2 * M + 1));
    uint64_t* Tq = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
    orc_mh_tables(alpha, L, M, w, q, Tq);
    int m[3] = {0, 0, 0};
    long acc = 0, tries = 0;
    int k = 0;
    for (uint64_t t = 0; k < K; ++t) {
        for (int a = 0; a < 3; ++a) {
            uint64_t blk[4];
            rng_block(seed, t, (uint64_t)a, 0, 4, blk);
            int mp = inv_cdf(blk[0], Tq, M);
            double u = (double)(blk[1] >> 11) * 1.1102230246251565e-16;
            double r = (w[mp + M] * q[m[a] + M]) / (w[m[a] + M] * q[mp + M]);
            ++tries;
            if (u < r) { m[a] = mp; ++acc; }
        }
        if (t < (uint64_t)burn) continue;
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) continue;
        pool[3 * k + 0] = m[0]; pool[3 * k + 1] = m[1]; pool[3 * k + 2] = m[2];
        ++k;
    }
    free(w); free(q); free(Tq);
    return (double)acc / (double)tries;
}

/* The P samples of a step under the parameters' sampling mode (R4 or R13). */
static void sample_k_mode(const orc_params* pr, uint64_t step, int32_t* m)
{
    if (pr->kpool <= 0) {
        orc_sample_k(pr->seed, step, pr->P, pr->alpha, pr->L, m);
        return;
    }
    int32_t* pool = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)pr->kpool);
    orc_kpool(pr->seed, pr->alpha, pr->L, pr->kpool, pr->kpool_burn, pool);
    for (int l = 0; l < pr->P; ++l) {
        uint64_t blk[4];
        rng_block(pr->seed, (uint64_t)l, 0, step, 5, blk);
        uint64_t e = uniform_below(blk[0], (uint64_t)pr->kpool);
        for (int a = 0; a < 3; ++a) m[3 * l + a] = pool[3 * e + a];
    }
    free(pool);
}

void orc_sample_k_params(const orc_params* pr, uint64_t step, int32_t* m) { sample_k_mode(pr, step, m); }

/* S = H^3 - 1 (Eq. (2.6)) with H by direct sum (Eq. (2.7), left side). */
double orc_S(double alpha, double L)
{
    int M = orc_kmax(alpha, L);
    uint64_t* T = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * M + 1));
    double H = orc_k_table(alpha, L, M, T);
    free(T);
    return H * H * H - 1.0;
}

/* ------------------------------------------------------------------------ */
/* Floyd sampling of p ordinals out of n (reading R3)                       */
/* ------------------------------------------------------------------------ */
/* words[k] is the 64-bit uniform for slot k; out[k] the ordinal chosen at
 * slot k (requires n > p). */
void orc_floyd(uint64_t n, int p, const uint64_t* words, uint64_t* out)
{
    for (int k = 0; k < p; ++k) {
        uint64_t j = n - (uint64_t)p + (uint64_t)k;
        uint64_t t = uniform_below(words[k], j + 1);
        int seen = 0;
        for (int l = 0; l < k; ++l)
            if (out[l] == t) { seen = 1; break; }
        out[k] = seen ? j : t;
    }
}

static void shell_words(uint64_t seed, uint64_t step, uint64_t atom, int p, uint64_t* words)
{
    for (int b = 0; 4 * b < p; ++b) {
        uint64_t w[4];
        rng_block(seed, atom, (uint64_t)b, step, 1, w);
        for (int q = 0; q < 4 && 4 * b + q < p; ++q) words[4 * b + q] = w[q];
    }
}

/* ------------------------------------------------------------------------ */
/* Neighbour sets C(i), S(i) in canonical order and the shell batch B(i)    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    const uint32_t* s;     /* [3n] fixed-point */
    const int32_t* cell;   /* [n] canonical linear cell */
    uint64_t Rc2, Rs2;
    int n_cell;
    /* cell lists (ascending atom id inside a cell) */
    const int32_t* cell_start; /* [n_cell^3 + 1] */
    const int32_t* cell_atoms; /* [n] */
} orc_grid;

/* Candidate enumeration in canonical order for atom i: either every atom
 * (brute force) or the distinct stencil cells of Sec. 2.3 (edge n_cell cells,
 * reach floor(r_s/w)+1 cells per axis), in ascending linear cell index. */
typedef struct {
    int count;
    int32_t* ids;
} cand_list;

static int add_axis_cells(int c, int reach, int nc, int* out)
{
    /* distinct cells within +-reach of c on a ring of nc, ascending */
    int k = 0;
    if (2 * reach + 1 >= nc) {
        for (int x = 0; x < nc; ++x) out[k++] = x;
        return k;
    }
    int mark[4096];
    int use_mark = nc <= 4096;
    if (use_mark) {
        for (int x = 0; x < nc; ++x) mark[x] = 0;
        for (int d = -reach; d <= reach; ++d) mark[((c + d) % nc + nc) % nc] = 1;
        for (int x = 0; x < nc; ++x) if (mark[x]) out[k++] = x;
        return k;
    }
    /* large grids: collect and sort the 2*reach+1 wrapped indices */
    for (int d = -reach; d <= reach; ++d) out[k++] = ((c + d) % nc + nc) % nc;
    for (int a = 1; a < k; ++a) {
        int v = out[a], b = a - 1;
        while (b >= 0 && out[b] > v) { out[b + 1] = out[b]; --b; }
        out[b + 1] = v;
    }
    return k;
}

/* Builds the canonical candidate list of atom i (cell mode). */
static void candidates_cells(const orc_grid* g, int i, int reach, cand_list* cl)
{
    int nc = g->n_cell;
    int ci = g->cell[i];
    int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
    int xs[4096], ys[4096], zs[4096];
    int nxs = add_axis_cells(cx, reach, nc, xs);
    int nys = add_axis_cells(cy, reach, nc, ys);
    int nzs = add_axis_cells(cz, reach, nc, zs);
    cl->count = 0;
    for (int a = 0; a < nzs; ++a)
        for (int b = 0; b < nys; ++b)
            for (int c = 0; c < nxs; ++c) {
                int lin = xs[c] + nc * (ys[b] + nc * zs[a]);
                for (int t = g->cell_start[lin]; t < g->cell_start[lin + 1]; ++t)
                    cl->ids[cl->count++] = g->cell_atoms[t];
            }
}

/* Per-atom list record. */
typedef struct {
    int n_core, n_shell, n_batch;
    int32_t* core;   /* ids in canonical order */
    int32_t* shell;  /* ids in canonical order */
    int32_t* batch;  /* ids of B(i) in slot order */
    int overlap;
} atom_lists;

/* Classify candidates (canonical order) into C(i) and S(i), then draw B(i). */
static void classify_and_sample(const orc_grid* g, int i, const int32_t* cand, int ncand,
                                int p, int shell_mode, uint64_t seed, uint64_t step, atom_lists* al,
                                uint64_t* words, uint64_t* ord)
{
    const uint32_t* si = g->s + 3 * i;
    al->n_core = 0; al->n_shell = 0; al->overlap = 0;
    for (int t = 0; t < ncand; ++t) {
        int j = cand[t];
        if (j == i) continue;
        uint64_t d2 = dist2_fixed(si, g->s + 3 * j);
        if (d2 == 0) al->overlap = 1;
        if (d2 <= g->Rc2) al->core[al->n_core++] = j;
        else if (d2 <= g->Rs2) al->shell[al->n_shell++] = j;
    }
    if (al->n_shell <= p) {
        for (int k = 0; k < al->n_shell; ++k) al->batch[k] = al->shell[k];
        al->n_batch = al->n_shell;
    } else {
        shell_words(seed, step, (uint64_t)i, p, words);
        if (shell_mode == 1) {
            /* R13: p independent uniform ordinals (with replacement) */
            for (int k = 0; k < p; ++k) ord[k] = uniform_below(words[k], (uint64_t)al->n_shell);
        } else {
            orc_floyd((uint64_t)al->n_shell, p, words, ord);
        }
        for (int k = 0; k < p; ++k) al->batch[k] = al->shell[ord[k]];
        al->n_batch = p;
    }
}

/* ------------------------------------------------------------------------ */
/* Pair term f_ij and u_ij (Eq. (2.10), readings R6, R7)                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double coul_pref;     /* k_e */
    double sqrt_alpha;
    double two_sqrt_alpha_over_sqrt_pi;
    double r_s;
    int shift_lj;
    double eps_ij[ORC_MAXT * ORC_MAXT];
    double sig_ij[ORC_MAXT * ORC_MAXT];
    double lj_shift[ORC_MAXT * ORC_MAXT];
    double lj_rc2[ORC_MAXT * ORC_MAXT];   /* squared LJ cutoff (R13)           */
    int lj_cut[ORC_MAXT * ORC_MAXT];      /* 1: cut at f sigma_ab < r_s (R13)  */
    int ntypes;
} pair_consts;

static void make_pair_consts(const orc_params* pr, pair_consts* pc)
{
    pc->coul_pref = pr->k_e;
    pc->sqrt_alpha = sqrt(pr->alpha);
    pc->two_sqrt_alpha_over_sqrt_pi = 2.0 * sqrt(pr->alpha) / sqrt(ORC_PI);
    pc->r_s = pr->r_s;
    pc->shift_lj = pr->shift_lj;
    pc->ntypes = pr->ntypes;
    for (int a = 0; a < pr->ntypes; ++a)
        for (int b = 0; b < pr->ntypes; ++b) {
            double e = sqrt(pr->eps[a] * pr->eps[b]);          /* Berthelot */
            double s = 0.5 * (pr->sigma[a] + pr->sigma[b]);    /* Lorentz   */
            pc->eps_ij[a * ORC_MAXT + b] = e;
            pc->sig_ij[a * ORC_MAXT + b] = s;
            /* R13: LJ cutoff min(f sigma_ab, r_s); the shift is U_LJ there */
            double rc = pr->r_s;
            int cut = 0;
            if (pr->lj_rc_factor > 0.0 && pr->lj_rc_factor * s < pr->r_s) {
                rc = pr->lj_rc_factor * s;
                cut = 1;
            }
            pc->lj_rc2[a * ORC_MAXT + b] = rc * rc;
            pc->lj_cut[a * ORC_MAXT + b] = cut;
            double sr6 = pow(s / rc, 6.0);
            pc->lj_shift[a * ORC_MAXT + b] = 4.0 * e * (sr6 * sr6 - sr6);
        }
}

/* Pair (i <- j) with displacement d = r_j - r_i (minimum image).
 * Returns the force on i (fx), and adds energies to u[0]=coul, u[1]=lj,
 * u[2]=exclusion, each multiplied by weight w. */
static void pair_term(const pair_consts* pc, double qi, double qj, int ti, int tj, int excluded,
                      const double d[3], double f[3], double u[3])
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double qq = pc->coul_pref * qi * qj;
    double gauss = pc->two_sqrt_alpha_over_sqrt_pi * exp(-(pc->sqrt_alpha * r) * (pc->sqrt_alpha * r));
    double s; /* f = s * d, i.e. the scalar multiplying r_ij */
    u[0] = u[1] = u[2] = 0.0;
    if (excluded) {
        /* u = -k_e q_i q_j erf(sqrt(a) r)/r ; F_i = (du/dr) d/r */
        double er = erf(pc->sqrt_alpha * r);
        double dudr = -qq * (gauss / r - er / r2);
        s = dudr / r;
        u[2] = -qq * er / r;
    } else {
        /* Eq. (2.10): -q_i q_j [erfc/r^2 + 2 sqrt(a) e^{-a r^2}/(sqrt(pi) r)] d/r */
        double ec = erfc(pc->sqrt_alpha * r);
        s = -qq * (ec / r2 + gauss / r) / r;
        u[0] = qq * ec / r;
        double e = pc->eps_ij[ti * ORC_MAXT + tj];
        int in_lj = !pc->lj_cut[ti * ORC_MAXT + tj] || r2 < pc->lj_rc2[ti * ORC_MAXT + tj];
        if (e != 0.0 && in_lj) {
            double sg = pc->sig_ij[ti * ORC_MAXT + tj];
            double sr2 = sg * sg / r2;
            double sr6 = sr2 * sr2 * sr2;
            /* Eq. (2.10) LJ: -eps (48 sig^12/r^14 - 24 sig^6/r^8) d */
            s += -e * (48.0 * sr6 * sr6 - 24.0 * sr6) / r2;
            u[1] = 4.0 * e * (sr6 * sr6 - sr6);
            if (pc->shift_lj) u[1] -= pc->lj_shift[ti * ORC_MAXT + tj];
        }
    }
    f[0] = s * d[0]; f[1] = s * d[1]; f[2] = s * d[2];
}

static void min_image(const double* ri, const double* rj, double L, double d[3])
{
    for (int a = 0; a < 3; ++a) {
        double x = rj[a] - ri[a];
        x -= L * round(x / L);
        d[a] = x;
    }
}

/* ------------------------------------------------------------------------ */
/* Grid construction                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t* s;
    int32_t* cell;
    int32_t* cell_start;
    int32_t* cell_atoms;
    int n_cell;
    int reach;
    uint64_t Rc2, Rs2;
} grid_storage;

static void build_grid(int n, const double* pos, const orc_params* pr, grid_storage* gs)
{
    double invL = 1.0 / pr->L;
    gs->n_cell = orc_n_cell(pr->L, pr->r_c);
    /* stencil reach floor(r_s / w) + 1 with w = L / n_cell (Sec. 2.3) */
    gs->reach = (int)floor(pr->r_s * (double)gs->n_cell / pr->L) + 1;
    gs->Rc2 = orc_radius2_fixed(pr->r_c, pr->L);
    gs->Rs2 = orc_radius2_fixed(pr->r_s, pr->L);
    int nc = gs->n_cell;
    long ncells = (long)nc * nc * nc;
    gs->s = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    gs->cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    gs->cell_start = (int32_t*)calloc((size_t)ncells + 1, sizeof(int32_t));
    gs->cell_atoms = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) gs->s[3 * i + a] = fixed_point(pos[3 * i + a], invL);
        uint32_t cx = cell_of(gs->s[3 * i + 0], nc);
        uint32_t cy = cell_of(gs->s[3 * i + 1], nc);
        uint32_t cz = cell_of(gs->s[3 * i + 2], nc);
        gs->cell[i] = (int32_t)(cx + (uint32_t)nc * (cy + (uint32_t)nc * cz));
        gs->cell_start[gs->cell[i] + 1] += 1;
    }
    for (long c = 0; c < ncells; ++c) gs->cell_start[c + 1] += gs->cell_start[c];
    int32_t* fill = (int32_t*)calloc((size_t)ncells, sizeof(int32_t));
    for (int i = 0; i < n; ++i) {
        int c = gs->cell[i];
        gs->cell_atoms[gs->cell_start[c] + fill[c]++] = i;
    }
    free(fill);
    /* R3: inside a cell, ascending (s_x, atom id) (insertion sort; ids are
     * already ascending, so equal s_x keep id order) */
    for (long c = 0; c < ncells; ++c) {
        int32_t* a = gs->cell_atoms + gs->cell_start[c];
        int cnt = gs->cell_start[c + 1] - gs->cell_start[c];
        for (int k = 1; k < cnt; ++k) {
            int32_t v = a[k];
            uint32_t key = gs->s[3 * v];
            int t = k - 1;
            while (t >= 0 && (gs->s[3 * a[t]] > key || (gs->s[3 * a[t]] == key && a[t] > v))) {
                a[t + 1] = a[t];
                --t;
            }
            a[t + 1] = v;
        }
    }
}

static void free_grid(grid_storage* gs)
{
    free(gs->s); free(gs->cell); free(gs->cell_start); free(gs->cell_atoms);
}

/* Canonical order of all atoms: ascending (cell, s_x, id) (R3). */
static void canonical_order(const grid_storage* gs, int n, int32_t* order)
{
    int nc = gs->n_cell;
    long ncells = (long)nc * nc * nc;
    int k = 0;
    for (long c = 0; c < ncells; ++c)
        for (int t = gs->cell_start[c]; t < gs->cell_start[c + 1]; ++t) order[k++] = gs->cell_atoms[t];
    (void)n;
}

/* ------------------------------------------------------------------------ */
/* Stored lists of the Verlet-skin variant (R15)                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    grid_storage gs;   /* grid of the rebuild step t_b */
    int32_t* order;    /* canonical order at t_b (brute-force enumeration) */
    int reach;         /* stencil reach for r_s + d */
    uint64_t Rv2;      /* floor(((r_s + d) 2^32 / L)^2) */
} skin_grid;

static void skin_grid_build(int n, const double* pos_b, const orc_params* pr, skin_grid* sg)
{
    build_grid(n, pos_b, pr, &sg->gs);
    double rv = pr->r_s + pr->skin;
    sg->reach = (int)floor(rv * (double)sg->gs.n_cell / pr->L) + 1;
    sg->Rv2 = orc_radius2_fixed(rv, pr->L);
    sg->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    canonical_order(&sg->gs, n, sg->order);
}

static void skin_grid_free(skin_grid* sg)
{
    free(sg->order);
    free_grid(&sg->gs);
}

/* V(i): candidates of the rebuild step in canonical order (the stencil for
 * r_s + d, or every atom when brute), kept when j != i and their exact
 * squared distance at t_b is at most Rv2.  tmp holds n ids. */
static void stored_list(const skin_grid* sg, int n, int i, int brute, int32_t* tmp, cand_list* out)
{
    const grid_storage* gs = &sg->gs;
    const int32_t* cand;
    int ncand;
    if (brute) {
        cand = sg->order;
        ncand = n;
    } else {
        orc_grid gb = {n, gs->s, gs->cell, gs->Rc2, gs->Rs2, gs->n_cell, gs->cell_start, gs->cell_atoms};
        cand_list c = {0, tmp};
        candidates_cells(&gb, i, sg->reach, &c);
        cand = tmp;
        ncand = c.count;
    }
    const uint32_t* si = gs->s + 3 * i;
    out->count = 0;
    for (int t = 0; t < ncand; ++t) {
        int j = cand[t];
        if (j == i) continue;
        if (dist2_fixed(si, gs->s + 3 * j) <= sg->Rv2) out->ids[out->count++] = j;
    }
}

/* R15 rebuild test: 1 when some atom moved, in fixed-point units, by more
 * than d/2 since the rebuild positions pos_b (sum of squared wrapped
 * differences above floor((d/2 2^32/L)^2)), else 0. */
int orc_skin_displaced(int n, const double* pos, const double* pos_b, double L, double skin)
{
    double invL = 1.0 / L;
    uint64_t D2 = orc_radius2_fixed(0.5 * skin, L);
    for (int i = 0; i < n; ++i) {
        uint32_t a[3], b[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = fixed_point(pos[3 * i + k], invL);
            b[k] = fixed_point(pos_b[3 * i + k], invL);
        }
        if (dist2_fixed(a, b) > D2) return 1;
    }
    return 0;
}

/* R15 stored lists themselves: counts[i] = |V(i)|, ids (cap per atom) in the
 * order of V(i); brute = 1 enumerates every atom instead of the stencil.
 * Returns 1 if some list exceeded cap, else 0. */
int orc_skin_lists(int n, const double* pos_b, const orc_params* pr, int brute, int32_t* counts, int32_t* ids,
                   int cap)
{
    skin_grid sg;
    skin_grid_build(n, pos_b, pr, &sg);
    int status = 0;
#pragma omp parallel
    {
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        cand_list v = {0, (int32_t*)malloc(sizeof(int32_t) * (size_t)n)};
        int local = 0;
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            stored_list(&sg, n, i, brute, tmp, &v);
            counts[i] = v.count;
            if (v.count > cap) local = 1;
            if (ids)
                for (int t = 0; t < v.count && t < cap; ++t) ids[(size_t)i * cap + t] = v.ids[t];
        }
#pragma omp critical
        status |= local;
        free(tmp); free(v.ids);
    }
    skin_grid_free(&sg);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Lists only (for bit-exact comparisons)                                   */
/* ------------------------------------------------------------------------ */
/* For every atom: n_core[i], n_shell[i], core ids (row-major, cap_core per
 * atom, canonical order), batch ids (cap_batch per atom, slot order), and
 * n_batch[i].  brute=1 enumerates all atoms, 0 uses the cell stencil.
 * Returns 0, or 1 if some list exceeded a cap, 2 on an r=0 overlap. */
static int lists_impl(int n, const double* pos, const double* pos_b, const orc_params* pr, uint64_t step, int brute,
                      int32_t* n_core, int32_t* n_shell, int32_t* n_batch,
                      int32_t* core, int cap_core, int32_t* batch, int cap_batch,
                      int32_t* shell, int cap_shell)
{
    grid_storage gs;
    build_grid(n, pos, pr, &gs);
    skin_grid sg;
    if (pos_b) skin_grid_build(n, pos_b, pr, &sg);
    orc_grid g = {n, gs.s, gs.cell, gs.Rc2, gs.Rs2, gs.n_cell, gs.cell_start, gs.cell_atoms};
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    canonical_order(&gs, n, order);
    int status = 0;
#pragma omp parallel
    {
        int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        atom_lists al;
        al.core = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        al.shell = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        al.batch = (int32_t*)malloc(sizeof(int32_t) * (size_t)(pr->p + 1));
        uint64_t* words = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(pr->p + 4));
        uint64_t* ord = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(pr->p + 4));
        int local_status = 0;
        cand_list v = {0, pos_b ? (int32_t*)malloc(sizeof(int32_t) * (size_t)n) : NULL};
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            int ncand;
            const int32_t* cl;
            if (pos_b) {
                /* R15: the members of V(i), in its order */
                stored_list(&sg, n, i, brute, cand, &v);
                cl = v.ids; ncand = v.count;
            } else if (brute) { cl = order; ncand = n; }
            else {
                cand_list c = {0, cand};
                candidates_cells(&g, i, gs.reach, &c);
                cl = cand; ncand = c.count;
            }
            classify_and_sample(&g, i, cl, ncand, pr->p, pr->shell_mode, pr->seed, step, &al, words, ord);
            n_core[i] = al.n_core; n_shell[i] = al.n_shell; n_batch[i] = al.n_batch;
            if (al.overlap) local_status |= 2;
            if (core) {
                if (al.n_core > cap_core) local_status |= 1;
                for (int t = 0; t < al.n_core && t < cap_core; ++t) core[(size_t)i * cap_core + t] = al.core[t];
            }
            if (shell) {
                if (al.n_shell > cap_shell) local_status |= 1;
                for (int t = 0; t < al.n_shell && t < cap_shell; ++t) shell[(size_t)i * cap_shell + t] = al.shell[t];
            }
            if (batch) {
                if (al.n_batch > cap_batch) local_status |= 1;
                for (int t = 0; t < al.n_batch && t < cap_batch; ++t) batch[(size_t)i * cap_batch + t] = al.batch[t];
            }
        }
#pragma omp critical
        status |= local_status;
        free(cand); free(al.core); free(al.shell); free(al.batch); free(words); free(ord); free(v.ids);
    }
    free(order);
    free_grid(&gs);
    if (pos_b) skin_grid_free(&sg);
    return status;
}

int orc_lists(int n, const double* pos, const orc_params* pr, uint64_t step, int brute,
              int32_t* n_core, int32_t* n_shell, int32_t* n_batch,
              int32_t* core, int cap_core, int32_t* batch, int cap_batch,
              int32_t* shell, int cap_shell)
{
    return lists_impl(n, pos, NULL, pr, step, brute, n_core, n_shell, n_batch, core, cap_core, batch, cap_batch,
                      shell, cap_shell);
}

/* R15: the lists of a step classified from the stored lists of the rebuild
 * positions pos_b (pr->skin > 0); brute = 1 builds V(i) from every atom. */
int orc_lists_skin(int n, const double* pos, const double* pos_b, const orc_params* pr, uint64_t step, int brute,
                   int32_t* n_core, int32_t* n_shell, int32_t* n_batch,
                   int32_t* core, int cap_core, int32_t* batch, int cap_batch,
                   int32_t* shell, int cap_shell)
{
    return lists_impl(n, pos, pos_b, pr, step, brute, n_core, n_shell, n_batch, core, cap_core, batch, cap_batch,
                      shell, cap_shell);
}

/* ------------------------------------------------------------------------ */
/* RBE Fourier part (Eq. (2.9), reading R8)                                  */
/* ------------------------------------------------------------------------ */
/* rho_l = sum_j q_j e^{i k_l . r_j} (Eq. (2.4)), k_l = 2 pi m_l / L. */
void orc_rho(int n, const double* pos, const double* q, double L, int P, const int32_t* m,
             double* rho /* [2P] re, im */)
{
    double twopi_L = 2.0 * ORC_PI / L;
#pragma omp parallel for schedule(static)
    for (int l = 0; l < P; ++l) {
        double kx = twopi_L * m[3 * l], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
        ksum re = {0, 0}, im = {0, 0};
        for (int j = 0; j < n; ++j) {
            double th = kx * pos[3 * j] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
            ksum_add(&re, q[j] * cos(th));
            ksum_add(&im, q[j] * sin(th));
        }
        rho[2 * l] = ksum_get(&re); rho[2 * l + 1] = ksum_get(&im);
    }
}

/* F_i^{long,*} = - sum_l (S/P) (4 pi k_e q_i k_l / (V k_l^2)) Im(e^{-i k_l.r_i} rho_l)
 * (Eq. (2.9)); energy and virial of the reweighted reciprocal sum. */
static void rbe_fourier(int n, const double* pos, const double* q, const orc_params* pr,
                        const int32_t* m, const double* rho, double* F, double* Fabs, double* Ek, double* Wk)
{
    double L = pr->L, V = L * L * L;
    double S = orc_S(pr->alpha, L);
    double twopi_L = 2.0 * ORC_PI / L;
    int P = pr->P;
    double* coef = (double*)malloc(sizeof(double) * (size_t)P);
    double E = 0.0, W[6] = {0, 0, 0, 0, 0, 0};
    for (int l = 0; l < P; ++l) {
        double kx = twopi_L * m[3 * l], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
        double k2 = kx * kx + ky * ky + kz * kz;
        coef[l] = (S / (double)P) * 4.0 * ORC_PI * pr->k_e / (V * k2);
        double rho2 = rho[2 * l] * rho[2 * l] + rho[2 * l + 1] * rho[2 * l + 1];
        double e = 0.5 * coef[l] * rho2;
        E += e;
        double b = 2.0 * (1.0 / k2 + 1.0 / (4.0 * pr->alpha));
        W[0] += e * (1.0 - b * kx * kx);
        W[1] += e * (1.0 - b * ky * ky);
        W[2] += e * (1.0 - b * kz * kz);
        W[3] += e * (-b * kx * ky);
        W[4] += e * (-b * kx * kz);
        W[5] += e * (-b * ky * kz);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double f[3] = {0, 0, 0}, fa[3] = {0, 0, 0};
        for (int l = 0; l < P; ++l) {
            double kx = twopi_L * m[3 * l], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
            double th = kx * pos[3 * i] + ky * pos[3 * i + 1] + kz * pos[3 * i + 2];
            /* Im(e^{-i th} rho) = cos(th) Im rho - sin(th) Re rho */
            double im = cos(th) * rho[2 * l + 1] - sin(th) * rho[2 * l];
            double g = -coef[l] * q[i] * im;
            f[0] += g * kx; f[1] += g * ky; f[2] += g * kz;
            double ga = coef[l] * fabs(q[i]) * (fabs(rho[2 * l]) + fabs(rho[2 * l + 1]));
            fa[0] += ga * fabs(kx); fa[1] += ga * fabs(ky); fa[2] += ga * fabs(kz);
        }
        F[3 * i] = f[0]; F[3 * i + 1] = f[1]; F[3 * i + 2] = f[2];
        Fabs[3 * i] = fa[0]; Fabs[3 * i + 1] = fa[1]; Fabs[3 * i + 2] = fa[2];
    }
    *Ek = E;
    for (int a = 0; a < 6; ++a) Wk[a] = W[a];
    free(coef);
}

/* ------------------------------------------------------------------------ */
/* The IRBE estimator (Algorithm 1, force steps; Eqs. (2.9)-(2.13))          */
/* ------------------------------------------------------------------------ */
/* Outputs: F[3n] total force, F_real[3n] (core + weighted shell, before the
 * momentum correction, may be NULL), F_long[3n] (may be NULL),
 * E[6] = {E_real_coul, E_k, E_self, E_lj, E_excl, 0}, W[6] = {xx,yy,zz,xy,xz,yz},
 * corr[3] the net-force correction of Eq. (2.12), m_out[3P] the k samples,
 * rho_out[2P], F_abs[3n] the sum of the absolute values of every summand
 * of each force component (pair terms, the correction, the k terms): the
 * scale that bounds the rounding error of the component.  mol may be NULL
 * (no exclusions); every output pointer may be NULL. */
static int rbe_forces_impl(int n, const double* pos, const double* pos_b, const double* q, const int32_t* type,
                           const int32_t* mol, const orc_params* pr, uint64_t step,
                           double* F, double* F_real_out, double* F_long_out, double* E, double* W,
                           double* corr, int32_t* m_out, double* rho_out, double* F_abs)
{
    grid_storage gs;
    build_grid(n, pos, pr, &gs);
    skin_grid sg;
    if (pos_b) skin_grid_build(n, pos_b, pr, &sg);
    orc_grid g = {n, gs.s, gs.cell, gs.Rc2, gs.Rs2, gs.n_cell, gs.cell_start, gs.cell_atoms};
    pair_consts pc;
    make_pair_consts(pr, &pc);
    double* Freal = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* Eat = (double*)malloc(sizeof(double) * 3 * (size_t)n);  /* coul, lj, excl per atom */
    double* Wat = (double*)malloc(sizeof(double) * 6 * (size_t)n);
    double* Aat = (double*)malloc(sizeof(double) * 3 * (size_t)n);  /* sum of |summands| */
    int status = 0;
#pragma omp parallel
    {
        int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        atom_lists al;
        al.core = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        al.shell = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        al.batch = (int32_t*)malloc(sizeof(int32_t) * (size_t)(pr->p + 1));
        uint64_t* words = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(pr->p + 4));
        uint64_t* ord = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(pr->p + 4));
        int local_status = 0;
        cand_list v = {0, pos_b ? (int32_t*)malloc(sizeof(int32_t) * (size_t)n) : NULL};
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            cand_list c = {0, cand};
            if (pos_b) {
                /* R15: the members of the stored list V(i), in its order */
                stored_list(&sg, n, i, 0, cand, &v);
                classify_and_sample(&g, i, v.ids, v.count, pr->p, pr->shell_mode, pr->seed, step, &al, words, ord);
            } else {
                candidates_cells(&g, i, gs.reach, &c);
                classify_and_sample(&g, i, cand, c.count, pr->p, pr->shell_mode, pr->seed, step, &al, words, ord);
            }
            if (al.overlap) local_status |= 2;
            double w_shell = (al.n_shell <= pr->p) ? 1.0 : (double)al.n_shell / (double)pr->p;
            double f[3] = {0, 0, 0}, u[3] = {0, 0, 0}, wv[6] = {0, 0, 0, 0, 0, 0}, fa[3] = {0, 0, 0};
            for (int part = 0; part < 2; ++part) {
                int cnt = part == 0 ? al.n_core : al.n_batch;
                const int32_t* ids = part == 0 ? al.core : al.batch;
                double w = part == 0 ? 1.0 : w_shell;
                for (int t = 0; t < cnt; ++t) {
                    int j = ids[t];
                    double d[3], fij[3], uij[3];
                    min_image(pos + 3 * i, pos + 3 * j, pr->L, d);
                    int excl = mol ? (mol[i] == mol[j]) : 0;
                    pair_term(&pc, q[i], q[j], type[i], type[j], excl, d, fij, uij);
                    for (int a = 0; a < 3; ++a) f[a] += w * fij[a];
                    for (int a = 0; a < 3; ++a) fa[a] += fabs(w * fij[a]);
                    for (int a = 0; a < 3; ++a) u[a] += w * uij[a];
                    wv[0] += w * d[0] * fij[0];
                    wv[1] += w * d[1] * fij[1];
                    wv[2] += w * d[2] * fij[2];
                    wv[3] += w * d[0] * fij[1];
                    wv[4] += w * d[0] * fij[2];
                    wv[5] += w * d[1] * fij[2];
                }
            }
            for (int a = 0; a < 3; ++a) Freal[3 * i + a] = f[a];
            for (int a = 0; a < 3; ++a) Aat[3 * i + a] = fa[a];
            for (int a = 0; a < 3; ++a) Eat[3 * i + a] = u[a];
            for (int a = 0; a < 6; ++a) Wat[6 * i + a] = wv[a];
        }
#pragma omp critical
        status |= local_status;
        free(cand); free(al.core); free(al.shell); free(al.batch); free(words); free(ord); free(v.ids);
    }
    if (pos_b) skin_grid_free(&sg);
    /* Eq. (2.12): net force of the real-space estimate (compensated sums) */
    double cr[3];
    for (int a = 0; a < 3; ++a) {
        ksum k = {0, 0};
        for (int i = 0; i < n; ++i) ksum_add(&k, Freal[3 * i + a]);
        cr[a] = ksum_get(&k) / (double)n;
    }
    double Ec, Elj, Ex, Wr[6];
    {
        ksum kc = {0, 0}, kl = {0, 0}, kx = {0, 0}, kw[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
        for (int i = 0; i < n; ++i) {
            ksum_add(&kc, Eat[3 * i]); ksum_add(&kl, Eat[3 * i + 1]); ksum_add(&kx, Eat[3 * i + 2]);
            for (int a = 0; a < 6; ++a) ksum_add(&kw[a], Wat[6 * i + a]);
        }
        Ec = ksum_get(&kc); Elj = ksum_get(&kl); Ex = ksum_get(&kx);
        for (int a = 0; a < 6; ++a) Wr[a] = ksum_get(&kw[a]);
    }
    /* Fourier part */
    int32_t* m = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)pr->P);
    double* rho = (double*)malloc(sizeof(double) * 2 * (size_t)pr->P);
    double* Flong = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* Flabs = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    sample_k_mode(pr, step, m);
    orc_rho(n, pos, q, pr->L, pr->P, m, rho);
    double Ek, Wk[6];
    rbe_fourier(n, pos, q, pr, m, rho, Flong, Flabs, &Ek, Wk);
    ksum kq2 = {0, 0};
    for (int i = 0; i < n; ++i) ksum_add(&kq2, q[i] * q[i]);
    double q2 = ksum_get(&kq2);
    /* Eq. (2.13) plus Eq. (2.9) */
    if (F)
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) F[3 * i + a] = Freal[3 * i + a] - cr[a] + Flong[3 * i + a];
    if (F_abs)
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) F_abs[3 * i + a] = Aat[3 * i + a] + fabs(cr[a]) + Flabs[3 * i + a];
    if (F_real_out) memcpy(F_real_out, Freal, sizeof(double) * 3 * (size_t)n);
    if (F_long_out) memcpy(F_long_out, Flong, sizeof(double) * 3 * (size_t)n);
    if (corr) for (int a = 0; a < 3; ++a) corr[a] = cr[a];
    if (E) {
        E[0] = 0.5 * Ec;
        E[1] = Ek;
        E[2] = -pr->k_e * sqrt(pr->alpha / ORC_PI) * q2;
        E[3] = 0.5 * Elj;
        E[4] = 0.5 * Ex;
        E[5] = 0.0;
    }
    if (W) for (int a = 0; a < 6; ++a) W[a] = -0.5 * Wr[a] + Wk[a];
    if (m_out) memcpy(m_out, m, sizeof(int32_t) * 3 * (size_t)pr->P);
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * 2 * (size_t)pr->P);
    free(m); free(rho); free(Flong); free(Flabs);
    free(Freal); free(Eat); free(Wat); free(Aat);
    free_grid(&gs);
    return status;
}

int orc_rbe_forces(int n, const double* pos, const double* q, const int32_t* type,
                   const int32_t* mol, const orc_params* pr, uint64_t step,
                   double* F, double* F_real_out, double* F_long_out, double* E, double* W,
                   double* corr, int32_t* m_out, double* rho_out, double* F_abs)
{
    return rbe_forces_impl(n, pos, NULL, q, type, mol, pr, step, F, F_real_out, F_long_out, E, W, corr, m_out,
                           rho_out, F_abs);
}

/* R15: the estimator of a step whose sets C(i), S(i) come from the stored
 * lists of the rebuild positions pos_b (pr->skin > 0). */
int orc_rbe_forces_skin(int n, const double* pos, const double* pos_b, const double* q, const int32_t* type,
                        const int32_t* mol, const orc_params* pr, uint64_t step,
                        double* F, double* F_real_out, double* F_long_out, double* E, double* W,
                        double* corr, int32_t* m_out, double* rho_out, double* F_abs)
{
    return rbe_forces_impl(n, pos, pos_b, q, type, mol, pr, step, F, F_real_out, F_long_out, E, W, corr, m_out,
                           rho_out, F_abs);
}

/* ------------------------------------------------------------------------ */
/* Exact reference sums (Eqs. (2.1), (2.3), (2.5))                          */
/* ------------------------------------------------------------------------ */
/* Ewald real space over all images with |r_ij + nL| <= r_cut (erfc term),
 * reciprocal space over all m != 0 with |m_a| <= kmax, self term, and the
 * exclusion correction for same-molecule pairs (minimum image).  LJ is the
 * brute-force minimum-image sum truncated at pr->r_s (pairs of one molecule
 * skipped).  E[6] as in orc_rbe_forces.  Returns 0. */
int orc_ewald_exact(int n, const double* pos, const double* q, const int32_t* type,
                    const int32_t* mol, const orc_params* pr, double r_cut, int kmax,
                    double* F, double* E, double* W)
{
    double L = pr->L, V = L * L * L;
    pair_consts pc;
    make_pair_consts(pr, &pc);
    int nimg = (int)ceil(r_cut / L);
    double* Fr = (double*)calloc(3 * (size_t)n, sizeof(double));
    double* Eat = (double*)calloc(3 * (size_t)n, sizeof(double));
    double* Wat = (double*)calloc(6 * (size_t)n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        double f[3] = {0, 0, 0}, u[3] = {0, 0, 0}, wv[6] = {0, 0, 0, 0, 0, 0};
        for (int j = 0; j < n; ++j) {
            int excl = mol ? (mol[i] == mol[j]) : 0;
            double d0[3];
            int n0[3];
            for (int a = 0; a < 3; ++a) {
                d0[a] = pos[3 * j + a] - pos[3 * i + a];
                n0[a] = -(int)round(d0[a] / L);   /* minimum-image shift */
            }
            for (int nx = -nimg; nx <= nimg; ++nx)
                for (int ny = -nimg; ny <= nimg; ++ny)
                    for (int nz = -nimg; nz <= nimg; ++nz) {
                        if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
                        /* an excluded pair's minimum image is replaced below */
                        if (excl && j != i && nx == n0[0] && ny == n0[1] && nz == n0[2]) continue;
                        double d[3] = {d0[0] + nx * L, d0[1] + ny * L, d0[2] + nz * L};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 > r_cut * r_cut) continue;
                        double r = sqrt(r2);
                        double qq = pr->k_e * q[i] * q[j];
                        double ec = erfc(pc.sqrt_alpha * r);
                        double gauss = pc.two_sqrt_alpha_over_sqrt_pi * exp(-pr->alpha * r2);
                        double s = -qq * (ec / r2 + gauss / r) / r;
                        u[0] += qq * ec / r;
                        double fv[3] = {s * d[0], s * d[1], s * d[2]};
                        for (int a = 0; a < 3; ++a) f[a] += fv[a];
                        wv[0] += d[0] * fv[0]; wv[1] += d[1] * fv[1]; wv[2] += d[2] * fv[2];
                        wv[3] += d[0] * fv[1]; wv[4] += d[0] * fv[2]; wv[5] += d[1] * fv[2];
                    }
            if (j == i) continue;
            double d[3], fij[3], uij[3];
            min_image(pos + 3 * i, pos + 3 * j, L, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (excl) {
                pair_term(&pc, q[i], q[j], type[i], type[j], 1, d, fij, uij);
                for (int a = 0; a < 3; ++a) f[a] += fij[a];
                u[2] += uij[2];
            } else if (r2 <= pr->r_s * pr->r_s) {
                /* LJ only: zero charge product isolates the LJ part */
                pair_term(&pc, 0.0, 0.0, type[i], type[j], 0, d, fij, uij);
                for (int a = 0; a < 3; ++a) f[a] += fij[a];
                u[1] += uij[1];
            } else {
                continue;
            }
            wv[0] += d[0] * fij[0]; wv[1] += d[1] * fij[1]; wv[2] += d[2] * fij[2];
            wv[3] += d[0] * fij[1]; wv[4] += d[0] * fij[2]; wv[5] += d[1] * fij[2];
        }
        for (int a = 0; a < 3; ++a) { Fr[3 * i + a] = f[a]; Eat[3 * i + a] = u[a]; }
        for (int a = 0; a < 6; ++a) Wat[6 * i + a] = wv[a];
    }
    double Ereal = 0, Elj = 0, Ex = 0, Wr[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        Ereal += Eat[3 * i]; Elj += Eat[3 * i + 1]; Ex += Eat[3 * i + 2];
        for (int a = 0; a < 6; ++a) Wr[a] += Wat[6 * i + a];
    }
    /* reciprocal space: enumerate m with m != 0, |m_a| <= kmax (Eq. (2.3)) */
    double twopi_L = 2.0 * ORC_PI / L;
    int side = 2 * kmax + 1;
    long nk = (long)side * side * side;
    double* Fk = (double*)calloc(3 * (size_t)n, sizeof(double));
    double Ek = 0.0, Wk[6] = {0, 0, 0, 0, 0, 0};
    /* rho(k) for every k, then per-atom forces */
    double* rre = (double*)malloc(sizeof(double) * (size_t)nk);
    double* rim = (double*)malloc(sizeof(double) * (size_t)nk);
#pragma omp parallel for schedule(dynamic, 64)
    for (long t = 0; t < nk; ++t) {
        int mx = (int)(t % side) - kmax, my = (int)((t / side) % side) - kmax, mz = (int)(t / ((long)side * side)) - kmax;
        double kx = twopi_L * mx, ky = twopi_L * my, kz = twopi_L * mz;
        double re = 0, im = 0;
        if (mx != 0 || my != 0 || mz != 0)
            for (int j = 0; j < n; ++j) {
                double th = kx * pos[3 * j] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
                re += q[j] * cos(th);
                im += q[j] * sin(th);
            }
        rre[t] = re; rim[t] = im;
    }
    for (long t = 0; t < nk; ++t) {
        int mx = (int)(t % side) - kmax, my = (int)((t / side) % side) - kmax, mz = (int)(t / ((long)side * side)) - kmax;
        if (mx == 0 && my == 0 && mz == 0) continue;
        double kx = twopi_L * mx, ky = twopi_L * my, kz = twopi_L * mz;
        double k2 = kx * kx + ky * ky + kz * kz;
        double e = (2.0 * ORC_PI * pr->k_e / (V * k2)) * exp(-k2 / (4.0 * pr->alpha)) *
                   (rre[t] * rre[t] + rim[t] * rim[t]);
        Ek += e;
        double b = 2.0 * (1.0 / k2 + 1.0 / (4.0 * pr->alpha));
        Wk[0] += e * (1.0 - b * kx * kx); Wk[1] += e * (1.0 - b * ky * ky); Wk[2] += e * (1.0 - b * kz * kz);
        Wk[3] += e * (-b * kx * ky); Wk[4] += e * (-b * kx * kz); Wk[5] += e * (-b * ky * kz);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double f[3] = {0, 0, 0};
        for (long t = 0; t < nk; ++t) {
            int mx = (int)(t % side) - kmax, my = (int)((t / side) % side) - kmax, mz = (int)(t / ((long)side * side)) - kmax;
            if (mx == 0 && my == 0 && mz == 0) continue;
            double kx = twopi_L * mx, ky = twopi_L * my, kz = twopi_L * mz;
            double k2 = kx * kx + ky * ky + kz * kz;
            double th = kx * pos[3 * i] + ky * pos[3 * i + 1] + kz * pos[3 * i + 2];
            double im = cos(th) * rim[t] - sin(th) * rre[t];
            /* Eq. (2.5), F^long */
            double g = -(4.0 * ORC_PI * pr->k_e * q[i] / (V * k2)) * exp(-k2 / (4.0 * pr->alpha)) * im;
            f[0] += g * kx; f[1] += g * ky; f[2] += g * kz;
        }
        for (int a = 0; a < 3; ++a) Fk[3 * i + a] = f[a];
    }
    double q2 = 0;
    for (int i = 0; i < n; ++i) q2 += q[i] * q[i];
    if (F) for (int i = 0; i < n; ++i) for (int a = 0; a < 3; ++a) F[3 * i + a] = Fr[3 * i + a] + Fk[3 * i + a];
    if (E) {
        E[0] = 0.5 * Ereal; E[1] = Ek; E[2] = -pr->k_e * sqrt(pr->alpha / ORC_PI) * q2;
        E[3] = 0.5 * Elj; E[4] = 0.5 * Ex; E[5] = 0.0;
    }
    if (W) for (int a = 0; a < 6; ++a) W[a] = -0.5 * Wr[a] + Wk[a];
    free(Fr); free(Eat); free(Wat); free(Fk); free(rre); free(rim);
    return 0;
}

/* Plain direct Coulomb lattice sum (Eq. (2.1), Coulomb part) over whole
 * image boxes with |n|_inf <= nshell, prime excluding i=j at n=0.  For a
 * neutral, dipole-free cell summed in cubic shells this converges to the
 * Ewald (tin-foil) value. */
double orc_direct_coulomb(int n, const double* pos, const double* q, double L, double k_e, int nshell)
{
    double U = 0.0;
    for (int nx = -nshell; nx <= nshell; ++nx)
        for (int ny = -nshell; ny <= nshell; ++ny)
            for (int nz = -nshell; nz <= nshell; ++nz)
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) {
                        if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
                        double d[3] = {pos[3 * j] - pos[3 * i] + nx * L, pos[3 * j + 1] - pos[3 * i + 1] + ny * L,
                                       pos[3 * j + 2] - pos[3 * i + 2] + nz * L};
                        U += q[i] * q[j] / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    }
    return 0.5 * k_e * U;
}

/* ------------------------------------------------------------------------ */
/* Bonded water terms and velocity Verlet (Algorithm 1, integration step)   */
/* ------------------------------------------------------------------------ */
/* Harmonic O-H bonds and H-O-H angle for molecules m = 0..nmol-1 whose atoms
 * are (first + 3m, +1, +2) = (O, H, H).  Adds forces to F and returns energy.
 * U = 1/2 kb (r - r0)^2 per bond, 1/2 kth (theta - th0)^2 per angle. */
double orc_water_bonded(int nmol, int first, const double* pos, double L, double kb, double r0,
                        double kth, double th0, double* F)
{
    double U = 0.0;
    for (int mI = 0; mI < nmol; ++mI) {
        int o = first + 3 * mI, h1 = o + 1, h2 = o + 2;
        double d1[3], d2[3];
        min_image(pos + 3 * o, pos + 3 * h1, L, d1);
        min_image(pos + 3 * o, pos + 3 * h2, L, d2);
        double r1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        double r2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
        /* bonds: F_h = -kb (r - r0) d/r, F_o = -F_h */
        double g1 = -kb * (r1 - r0) / r1, g2 = -kb * (r2 - r0) / r2;
        U += 0.5 * kb * (r1 - r0) * (r1 - r0) + 0.5 * kb * (r2 - r0) * (r2 - r0);
        for (int a = 0; a < 3; ++a) {
            F[3 * h1 + a] += g1 * d1[a];
            F[3 * o + a] -= g1 * d1[a];
            F[3 * h2 + a] += g2 * d2[a];
            F[3 * o + a] -= g2 * d2[a];
        }
        /* angle: theta = acos(d1.d2 / (r1 r2)) */
        double c = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (r1 * r2);
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        double th = acos(c);
        double sn = sqrt(1.0 - c * c);
        if (sn < 1e-12) sn = 1e-12;
        U += 0.5 * kth * (th - th0) * (th - th0);
        /* dU/dtheta = kth (th - th0); dtheta/dd1 = -(d2/(r1 r2) - c d1/r1^2)/sin */
        double dUdth = kth * (th - th0);
        for (int a = 0; a < 3; ++a) {
            double dth_dd1 = -(d2[a] / (r1 * r2) - c * d1[a] / (r1 * r1)) / sn;
            double dth_dd2 = -(d1[a] / (r1 * r2) - c * d2[a] / (r2 * r2)) / sn;
            double f1 = -dUdth * dth_dd1, f2 = -dUdth * dth_dd2;
            F[3 * h1 + a] += f1;
            F[3 * h2 + a] += f2;
            F[3 * o + a] -= f1 + f2;
        }
    }
    return U;
}

/* Velocity Verlet: nsteps of  v += F dt/(2m) a; x += v dt; F = F(x, step+1);
 * v += F dt/(2m) a  with a = accel (force-to-acceleration unit factor).
 * F holds the forces at (pos, step0) on entry and at the final positions on
 * exit.  etrace[2*k] = potential (sum of E[0..5]), etrace[2*k+1] = kinetic
 * after step k.  Water bonds are applied when nmol_w > 0 (atoms 0..3*nmol_w-1). */
/* Langevin force of R14 at step s from the current velocities (FL = 0 when
 * the thermostat is off). */
static void langevin_force(int n, const double* vel, const double* mass, const orc_params* pr, uint64_t s,
                           double dt, double accel, double* FL)
{
    if (!(pr->lang_tau > 0.0)) {
        for (int i = 0; i < 3 * n; ++i) FL[i] = 0.0;
        return;
    }
    double c1 = accel * pr->lang_tau;                   /* m / c1: friction coefficient */
    double c2 = 24.0 * pr->lang_kT / (c1 * dt);         /* sqrt(m c2): noise amplitude  */
    for (int i = 0; i < n; ++i) {
        uint64_t w[4];
        rng_block(pr->seed, (uint64_t)i, 0, s, 3, w);
        double amp = sqrt(mass[i] * c2);
        for (int a = 0; a < 3; ++a) {
            double u = (double)(w[a] >> 11) * 1.1102230246251565e-16;
            FL[3 * i + a] = -(mass[i] / c1) * vel[3 * i + a] + amp * (u - 0.5);
        }
    }
}

int orc_vv_run(int n, double* pos, double* vel, const double* mass, const double* q,
               const int32_t* type, const int32_t* mol, const orc_params* pr,
               uint64_t step0, int nsteps, double dt, double accel,
               int nmol_w, double kb, double r0, double kth, double th0,
               double* F, double* etrace)
{
    double E[6], W[6];
    int status = 0;
    double* FL = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    langevin_force(n, vel, mass, pr, step0, dt, accel, FL);
    for (int k = 0; k < nsteps; ++k) {
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a)
                vel[3 * i + a] += 0.5 * dt * accel * (F[3 * i + a] + FL[3 * i + a]) / mass[i];
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) pos[3 * i + a] += dt * vel[3 * i + a];
        status |= orc_rbe_forces(n, pos, q, type, mol, pr, step0 + (uint64_t)k + 1, F, NULL, NULL, E, W,
                                 NULL, NULL, NULL, NULL);
        if (nmol_w > 0) E[5] = orc_water_bonded(nmol_w, 0, pos, pr->L, kb, r0, kth, th0, F);
        langevin_force(n, vel, mass, pr, step0 + (uint64_t)k + 1, dt, accel, FL);
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a)
                vel[3 * i + a] += 0.5 * dt * accel * (F[3 * i + a] + FL[3 * i + a]) / mass[i];
        if (etrace) {
            double ke = 0.0;
            for (int i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) ke += 0.5 * mass[i] * vel[3 * i + a] * vel[3 * i + a];
            etrace[2 * k] = E[0] + E[1] + E[2] + E[3] + E[4] + E[5];
            etrace[2 * k + 1] = ke / accel;
        }
    }
    free(FL);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Gradients of the estimator with frozen draws (derivatives of R8 and of   */
/* Eqs. (2.9)-(2.13) with respect to charges and LJ pair parameters)        */
/* ------------------------------------------------------------------------ */
/* For the estimator energy E = sum of E[0..4] and the force functional
 * L = sum_i v_i . F_i (v = gF, may be NULL) at fixed (seed, step):
 *   dEdq[n], dLdq[n]                      gradient w.r.t. each charge;
 *   dEde[T*T], dEds[T*T], dLde, dLds     gradient w.r.t. the mixed pair
 *       parameters eps_ab, sigma_ab of the ordered type pair (a, b) = (t_i, t_j)
 *       of each pair term (T = ORC_MAXT row stride).
 * Lists and draws are those of orc_rbe_forces at the same step.  The momentum
 * correction enters L through the centred v_i - mean(v) on the real-space
 * force (Eq. (2.13)); the Fourier part uses
 *   tau_l = sum_i q_i (v_i . k_l) exp(i k_l . r_i). */
int orc_rbe_adjoint(int n, const double* pos, const double* q, const int32_t* type, const int32_t* mol,
                    const orc_params* pr, uint64_t step, const double* gF,
                    double* dEdq, double* dLdq, double* dEde, double* dEds, double* dLde, double* dLds)
{
    grid_storage gs;
    build_grid(n, pos, pr, &gs);
    orc_grid g = {n, gs.s, gs.cell, gs.Rc2, gs.Rs2, gs.n_cell, gs.cell_start, gs.cell_atoms};
    pair_consts pc;
    make_pair_consts(pr, &pc);
    const int T = ORC_MAXT;
    double vbar[3] = {0, 0, 0};
    if (gF) {
        for (int a = 0; a < 3; ++a) {
            ksum k = {0, 0};
            for (int i = 0; i < n; ++i) ksum_add(&k, gF[3 * i + a]);
            vbar[a] = ksum_get(&k) / (double)n;
        }
    }
    /* per ordered pair contributions, accumulated per atom i (own part) and
     * per (i, slot) for the transposed part, then summed sequentially */
    double* own_E = (double*)calloc((size_t)n, sizeof(double));
    double* own_L = (double*)calloc((size_t)n, sizeof(double));
    typedef struct { int j; double cE, cL; } tr_rec;
    int cap_tr = 1024;
    tr_rec* tr = (tr_rec*)malloc(sizeof(tr_rec) * (size_t)n * (size_t)cap_tr);
    int* ntr = (int*)calloc((size_t)n, sizeof(int));
    double* lj_at = (double*)calloc((size_t)n * 4 * T * T, sizeof(double)); /* per atom: dEde dEds dLde dLds */
    int status = 0;
#pragma omp parallel
    {
        int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        atom_lists al;
        al.core = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        al.shell = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        al.batch = (int32_t*)malloc(sizeof(int32_t) * (size_t)(pr->p + 1));
        uint64_t* words = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(pr->p + 4));
        uint64_t* ord = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(pr->p + 4));
        int local_status = 0;
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            cand_list c = {0, cand};
            candidates_cells(&g, i, gs.reach, &c);
            classify_and_sample(&g, i, cand, c.count, pr->p, pr->shell_mode, pr->seed, step, &al, words, ord);
            double w_shell = (al.n_shell <= pr->p) ? 1.0 : (double)al.n_shell / (double)pr->p;
            double vt[3] = {0, 0, 0};
            if (gF) for (int a = 0; a < 3; ++a) vt[a] = gF[3 * i + a] - vbar[a];
            double* lj = lj_at + (size_t)i * 4 * T * T;
            for (int part = 0; part < 2; ++part) {
                int cnt = part == 0 ? al.n_core : al.n_batch;
                const int32_t* ids = part == 0 ? al.core : al.batch;
                double w = part == 0 ? 1.0 : w_shell;
                for (int t = 0; t < cnt; ++t) {
                    int j = ids[t];
                    double d[3];
                    min_image(pos + 3 * i, pos + 3 * j, pr->L, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    double r = sqrt(r2);
                    int excl = mol ? (mol[i] == mol[j]) : 0;
                    double ar = pc.sqrt_alpha * r;
                    double gauss = pc.two_sqrt_alpha_over_sqrt_pi * exp(-ar * ar);
                    /* Coulomb kernel per unit k_e q_i q_j: energy phi, force h d */
                    double phi, h;
                    if (excl) {
                        double er = erf(ar);
                        phi = -er / r;
                        h = -(gauss / r - er / r2) / r;
                    } else {
                        double ec = erfc(ar);
                        phi = ec / r;
                        h = -(ec / r2 + gauss / r) / r;
                    }
                    double vd = vt[0] * d[0] + vt[1] * d[1] + vt[2] * d[2];
                    double ke = pc.coul_pref;
                    /* own part (derivative w.r.t. q_i) */
                    own_E[i] += 0.5 * w * ke * q[j] * phi;
                    own_L[i] += w * ke * q[j] * h * vd;
                    /* transposed part (derivative w.r.t. q_j) */
                    if (ntr[i] < cap_tr) {
                        tr[(size_t)i * cap_tr + ntr[i]].j = j;
                        tr[(size_t)i * cap_tr + ntr[i]].cE = 0.5 * w * ke * q[i] * phi;
                        tr[(size_t)i * cap_tr + ntr[i]].cL = w * ke * q[i] * h * vd;
                        ntr[i]++;
                    } else {
                        local_status |= 1;
                    }
                    /* LJ pair parameters */
                    int tti = type[i] * ORC_MAXT + type[j];
                    if (!excl && (!pc.lj_cut[tti] || r2 < pc.lj_rc2[tti])) {
                        int ti = type[i], tj = type[j];
                        double e = pc.eps_ij[ti * ORC_MAXT + tj], sg = pc.sig_ij[ti * ORC_MAXT + tj];
                        double sr = sg / r, sr6 = pow(sr, 6.0), sr12 = sr6 * sr6;
                        /* u = 4 e (sr12 - sr6) - shift ; h_lj d with h_lj = -e (48 sg^12/r^14 - 24 sg^6/r^8) */
                        double du_de = 4.0 * (sr12 - sr6);
                        double du_ds = 4.0 * e * (12.0 * sr12 - 6.0 * sr6) / sg;
                        if (pc.shift_lj) {
                            /* shift 4 e ((sg/rc)^12 - (sg/rc)^6): with rc = f sg
                             * (R13) it does not depend on sg */
                            double rc = pc.lj_cut[tti] ? sqrt(pc.lj_rc2[tti]) : pc.r_s;
                            double ss = sg / rc, ss6 = pow(ss, 6.0), ss12 = ss6 * ss6;
                            du_de -= 4.0 * (ss12 - ss6);
                            if (!pc.lj_cut[tti]) du_ds -= 4.0 * e * (12.0 * ss12 - 6.0 * ss6) / sg;
                        }
                        double dh_de = -(48.0 * sr12 - 24.0 * sr6) / r2;
                        double dh_ds = -e * (576.0 * sr12 - 144.0 * sr6) / (r2 * sg);
                        int k = ti * T + tj;
                        lj[0 * T * T + k] += 0.5 * w * du_de;
                        lj[1 * T * T + k] += 0.5 * w * du_ds;
                        lj[2 * T * T + k] += w * dh_de * vd;
                        lj[3 * T * T + k] += w * dh_ds * vd;
                    }
                }
            }
        }
#pragma omp critical
        status |= local_status;
        free(cand); free(al.core); free(al.shell); free(al.batch); free(words); free(ord);
    }
    /* Fourier part */
    int32_t* m = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)pr->P);
    double* rho = (double*)malloc(sizeof(double) * 2 * (size_t)pr->P);
    double* tau = (double*)calloc(2 * (size_t)pr->P, sizeof(double));
    sample_k_mode(pr, step, m);
    orc_rho(n, pos, q, pr->L, pr->P, m, rho);
    double L = pr->L, V = L * L * L;
    double S = orc_S(pr->alpha, L);
    double twopi_L = 2.0 * ORC_PI / L;
    if (gF) {
#pragma omp parallel for schedule(static)
        for (int l = 0; l < pr->P; ++l) {
            double kx = twopi_L * m[3 * l], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
            ksum re = {0, 0}, im = {0, 0};
            for (int i = 0; i < n; ++i) {
                double th = kx * pos[3 * i] + ky * pos[3 * i + 1] + kz * pos[3 * i + 2];
                double vk = gF[3 * i] * kx + gF[3 * i + 1] * ky + gF[3 * i + 2] * kz;
                ksum_add(&re, q[i] * vk * cos(th));
                ksum_add(&im, q[i] * vk * sin(th));
            }
            tau[2 * l] = ksum_get(&re);
            tau[2 * l + 1] = ksum_get(&im);
        }
    }
    double self = -2.0 * pr->k_e * sqrt(pr->alpha / ORC_PI);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double gE = 0.0, gL = 0.0;
        for (int l = 0; l < pr->P; ++l) {
            double kx = twopi_L * m[3 * l], ky = twopi_L * m[3 * l + 1], kz = twopi_L * m[3 * l + 2];
            double k2 = kx * kx + ky * ky + kz * kz;
            double c = (S / (double)pr->P) * 4.0 * ORC_PI * pr->k_e / (V * k2);
            double th = kx * pos[3 * i] + ky * pos[3 * i + 1] + kz * pos[3 * i + 2];
            double cs = cos(th), sn = sin(th);
            /* dE_k/dq_i = sum_l c_l Re(conj(rho_l) e^{i th}) */
            gE += c * (rho[2 * l] * cs + rho[2 * l + 1] * sn);
            if (gF) {
                double vk = gF[3 * i] * kx + gF[3 * i + 1] * ky + gF[3 * i + 2] * kz;
                /* Im(e^{-i th} rho) and Im(e^{i th} conj(tau)) */
                double im1 = cs * rho[2 * l + 1] - sn * rho[2 * l];
                double im2 = sn * tau[2 * l] - cs * tau[2 * l + 1];
                gL += -c * (vk * im1 + im2);
            }
        }
        if (dEdq) dEdq[i] = gE + self * q[i];
        if (dLdq) dLdq[i] = gL;
    }
    /* pair parts: own then transposed, sequential over atoms */
    for (int i = 0; i < n; ++i) {
        if (dEdq) dEdq[i] += own_E[i];
        if (dLdq) dLdq[i] += own_L[i];
    }
    for (int i = 0; i < n; ++i)
        for (int t = 0; t < ntr[i]; ++t) {
            const tr_rec* rcd = tr + (size_t)i * cap_tr + t;
            if (dEdq) dEdq[rcd->j] += rcd->cE;
            if (dLdq) dLdq[rcd->j] += rcd->cL;
        }
    double* outs[4] = {dEde, dEds, dLde, dLds};
    for (int o = 0; o < 4; ++o) {
        if (!outs[o]) continue;
        for (int k = 0; k < T * T; ++k) {
            ksum s = {0, 0};
            for (int i = 0; i < n; ++i) ksum_add(&s, lj_at[(size_t)i * 4 * T * T + (size_t)o * T * T + k]);
            outs[o][k] = ksum_get(&s);
        }
    }
    free(own_E); free(own_L); free(tr); free(ntr); free(lj_at);
    free(m); free(rho); free(tau);
    free_grid(&gs);
    return status;
}
