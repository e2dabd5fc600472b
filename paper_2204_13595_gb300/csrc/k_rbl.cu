// k_rbl.cu -- random batch list (RBL) real-space kernel, Sec. 2.3.
//
// Work unit = the atoms of G consecutive cells of one x-row of the cell grid
// (cells of edge L/floor(L/r_c), the grid of Sec. 2.3).  A block takes units
// round-robin; for each unit it stages, in shared memory, the FP32 positions
// of every atom in the union of the unit's stencils: (2R+1)^2 rows of G+2R
// cells, R = floor(r_s/w)+1 (Sec. 2.3's stencil reach), by one bulk
// asynchronous copy per contiguous piece of a row (completing on an
// mbarrier), each piece that lies across the box boundary then moved to the
// periodic image adjacent to the unit.  Each warp then owns one atom i of the
// unit at a time (two atoms A, B of the same cell row on the mixed path,
// which share the range lookups and staged loads of the classification and
// split the warp's lanes between their pair terms):
//   1. list construction: the lanes take i's stencil rows (32 per pass) in
//      canonical order (ascending wrapped cell index, then fixed-point x, then
//      atom index); each row is cut to the cells that can hold a point within
//      r_s and, by binary search on the x-sorted end cells, to the atoms
//      within the row's x half-width, leaving one or two contiguous ranges of
//      the staged array.  The ranges of a pass are concatenated in canonical
//      order and classified 32 candidates per lane-chunk, four chunks at a
//      time, into the core C(i) (r <= r_c) and the shell S(i)
//      (r_c < r <= r_s) by an FP32 distance whose rounding is bounded on the
//      host; candidates inside that bound of r_c or r_s, and r ~ 0, are
//      decided by the exact integer squared distance of the 32-bit fixed-point
//      coordinates, so the sets equal the exact-integer definition bit for
//      bit.  Members are appended in order to per-warp shared buffers (ballot
//      + popc ranks).
//   2. shell batch: if N_S > p, Floyd's algorithm draws p distinct ordinals
//      in [0, N_S) from Philox words at counter (i, k/4, step, 1); otherwise
//      the batch is all of S(i) with weight 1 (Algorithm 1, shell step).
//   3. pair terms f_ij of Eq. (2.10) over C(i) (weight 1) and B(i) (weight
//      N_S/p, Eq. (2.11)); same-molecule pairs take the Ewald exclusion
//      correction instead of erfc + LJ.
// A unit whose staged region exceeds the shared capacity reads the same
// ranges from global memory one range at a time, and so does a pass whose
// concatenated ranges hold more than RBL_MAX_PACKED candidates (identical
// results, slower).
// Outputs: F_real (core + weighted shell, before the momentum correction of
// Eq. (2.13)) per sorted atom -- FP64 on the FP64 path, FP32 on the mixed
// path -- and per-block partial sums of the real-space energies, the virial
// and the net force in a fixed order.
#include <math.h>
#include <string.h>

#include "rbe_internal.cuh"

namespace {

constexpr int WARPS = RBE_WARPS_RBL;

struct RblArgs {
    int n;
    uint64_t step;
    const uint4* __restrict__ s4;
    const float4* __restrict__ f4;
    const double4_32a* __restrict__ p4;
    const int2* __restrict__ tm;
    const int* __restrict__ perm;
    const int* __restrict__ cell_start;
    const RbeLJ* __restrict__ lj;
    double* __restrict__ F_real;
    double* __restrict__ part;
    int* __restrict__ status;
    RbeConsts c;
    RblGeom g;
    int core_cap, shell_cap;
    int nslots;                          // blocks (slots) of the replica's grid
    int debug, dbg_cap;
    // adjoint mode
    const double* __restrict__ vs;       // [3n] upstream gradient, sorted
    const double* __restrict__ vbar;     // [3] its mean
    double* __restrict__ gq_own;         // [2n]
    double* __restrict__ gq_tr;          // [2n]
    double* __restrict__ part_lj;        // [grid * 4 * nt2]
    int* __restrict__ dbg_ncore;
    int* __restrict__ dbg_nshell;
    int* __restrict__ dbg_core;
    int* __restrict__ dbg_batch;
    int* __restrict__ dbg_unstaged;
    // Verlet skin (stored lists): V(i) of sorted atom i at vlist[i * vcap ..],
    // its length at vcnt[i]
    int* __restrict__ vlist;
    int* __restrict__ vcnt;
    int vcap;
};

// Modes of the pair kernel: the stencil walk of every step; the stencil walk
// at r_s + skin that writes the stored lists V(i) of the Verlet-skin variant
// (no batches, no pair terms); the classification of the stored lists at
// the current positions followed by the batches and pair terms.
constexpr int RBL_STENCIL = 0;
constexpr int RBL_BUILD = 1;
constexpr int RBL_STORED = 2;

// Per-row description of the staged region of the current unit (64 bytes).
struct __align__(16) RowInfo {
    int zc, yc;            // wrapped cell coordinates of the row
    float shy, shz;        // periodic image shift of the row (0 or +-L)
    int sbase;             // first staged slot of the row
    int ul;                // first unwrapped x cell staged
    int goff[3];           // global - staged index offset for u < 0, 0 <= u < nc, u >= nc
    float zs, ys;          // sign of the row's z / y cell offset from the unit
    float zb, yb;          // slab boundary (fraction of L) giving the yz gap
    int pad;
};
static_assert(sizeof(RowInfo) == 64, "RowInfo layout");

// Candidate ranges of one pass of 32 stencil rows: at most two per row.  A
// pass whose concatenated ranges hold more than RBL_MAX_PACKED candidates is
// walked range by range instead.
constexpr int RBL_MAX_RANGES = 64;
constexpr int RBL_MAX_PACKED = 2048;
// Words of the per-warp shell buffer used by the two-atom path beyond B's
// core list: shell ballot words [2 * 64], their prefix counts for A and B
// and the range-start prefix [3 * 64], the batches of A and B [2 * 32] and
// B's slot ordinals [32]
constexpr int RBL_PAIR_CARVE = 2 * 64 + 3 * 64 + 3 * 32;
static_assert(RBL_PAIR_CARVE == RBE_RBL_PAIR_CARVE, "carve of the two-atom path");

// Shared-memory layout of k_rbl; every section starts on a 16-byte boundary.
// Per warp: the range table of the current pass [RBL_MAX_RANGES] int2 and the
// bitmap of range starts [RBL_MAX_PACKED / 32] words, the Philox words
// [ga][p_pad], the core and shell lists and the batch ordinals, and (stored-
// list kernel only) the double buffer of stored-list entries [2][RBL_LGROUP].
struct SmemLayout {
    size_t rows, cellpos, cellabs, lj, warps, wbytes, lbuf, total;
    int ga;                // atoms whose Philox words are made in one warp pass
};
// entries of a stored list V(i) classified per step of the stored-list
// kernel (four chunks of 32), copied one step ahead
constexpr int RBL_LGROUP = 128;

__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline SmemLayout smem_layout(const RblGeom& g, int nt2, int p, int core_cap, int shell_cap,
                                                  bool list_buffer = false)
{
    SmemLayout L;
    const int p_pad = (p + 3) & ~3;
    const int nbk = p_pad / 4;
    L.ga = nbk >= 32 ? 1 : 32 / nbk;
    size_t o = up16(sizeof(float4) * (size_t)g.cap_stage);
    L.rows = o;
    o = up16(o + sizeof(RowInfo) * (size_t)g.nrows);
    L.cellpos = o;
    o = up16(o + sizeof(int) * (size_t)g.nrows * (size_t)(g.cells_per_row + 1));
    L.cellabs = o;
    o = up16(o + sizeof(int) * (size_t)g.nrows * (size_t)(g.cells_per_row + 1));
    L.lj = o;
    o = up16(o + sizeof(double) * 12 * (size_t)nt2);
    L.warps = o;
    L.wbytes = sizeof(int2) * RBL_MAX_RANGES + sizeof(unsigned) * (RBL_MAX_PACKED / 32) +
               up16(sizeof(uint64_t) * (size_t)p_pad * L.ga + sizeof(int) * (size_t)(core_cap + shell_cap + p_pad));
    L.lbuf = L.wbytes;     // offset inside a warp's region
    if (list_buffer) L.wbytes += sizeof(int) * 2 * RBL_LGROUP;
    L.total = o + L.wbytes * WARPS;
    return L;
}

__device__ __forceinline__ int wrapc(int u, int nc) { return u < 0 ? u + nc : (u >= nc ? u - nc : u); }

// Unwrapped coordinate of the k-th stencil row around cell c in ascending
// wrapped order (ring of nc cells, 2R+1 < nc distinct rows).
__device__ __forceinline__ int ring_row(int k, int c, int R, int nc)
{
    int lo = c - R;
    int w = (lo < 0) ? ((k <= c + R) ? k : lo + nc + (k - (c + R + 1)))
                     : ((c + R >= nc) ? ((k <= c + R - nc) ? k : lo + (k - (c + R - nc + 1))) : lo + k);
    int d = w - c;
    if (d > R) d -= nc;
    if (d < -R) d += nc;
    return c + d;
}

// Exact squared distance of the fixed-point codes (reading of the sets C, S).
__device__ __forceinline__ unsigned long long d2_exact(uint4 a, uint4 b)
{
    int dx = (int)(b.x - a.x), dy = (int)(b.y - a.y), dz = (int)(b.z - a.z);
    return (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
           (unsigned long long)((long long)dz * dz);
}


// Trim the canonical segment [b, e) of a stencil row to the atoms whose x lies
// within [xref - H, xref + H]: inside a cell atoms are sorted by their
// fixed-point x code, so the staged FP32 x is non-decreasing there (up to one
// ulp between atoms of equal code) and the first and last cells of the
// segment are cut by binary search.  H = hx L is the row's x half-width
// bound already used to choose the segment's cells (conservative by
// construction: every member of C or S has |dx| <= r_s < H - 1e-3 A), so no
// member is dropped and the exact classification is unchanged.
__device__ __forceinline__ void trim_range(const float4* __restrict__ src, int& b, int& e, int cnt_lo, int cnt_hi,
                                           bool one_cell, float lo_x, float hi_x)
{
    // the lower cut (first x >= lo_x in the first cell) and the upper cut
    // (first x > hi_x in the last cell) are independent searches, run
    // together so that their shared-memory loads overlap
    int l = b, r = b + cnt_lo;
    int l2 = one_cell ? b : e - cnt_hi, r2 = e;
    while (l < r || l2 < r2) {
        const int m = (l + r) >> 1, m2 = (l2 + r2) >> 1;
        const float xa = l < r ? src[m].x : 0.f;
        const float xb = l2 < r2 ? src[m2].x : 0.f;
        if (l < r) {
            if (xa < lo_x) l = m + 1;
            else r = m;
        }
        if (l2 < r2) {
            if (xb <= hi_x) l2 = m2 + 1;
            else r2 = m2;
        }
    }
    b = l;
    e = l2 < l ? l : l2;
}

__device__ __forceinline__ void trim_segment(const float4* __restrict__ src, int& b, int& e, int cnt_lo, int cnt_hi,
                                             bool one_cell, float xref, float H)
{
    trim_range(src, b, e, cnt_lo, cnt_hi, one_cell, xref - H, xref + H);
}

// erfc(x) for x >= 0 in FP32 by Hastings' approximation (Abramowitz & Stegun,
// Handbook of Mathematical Functions, 7.1.26): erfc x = t (a1 + t (a2 + t (a3
// + t (a4 + t a5)))) e^{-x^2}, t = 1 / (1 + p x), with absolute error below
// 1.5e-7 for every x >= 0.  ex2 = e^{-x^2} is passed in: the pair force needs
// it anyway.  Branch free, unlike a general erfc, whose argument ranges make
// the lanes of a warp diverge.
__device__ __forceinline__ float erfc_hastings(float x, float ex2)
{
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    const float poly = fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                            0.254829592f);
    return t * poly * ex2;
}

// erf(x) (want_erf) or erfc(x) for x >= 0 in FP64 by W. J. Cody's rational
// Chebyshev approximations (Math. Comp. 23 (1969) 631-637, the intervals
// [0, 0.46875], (0.46875, 4] and (4, inf)): erf = x R1(x^2) on the first,
// erfc = e^{-x^2} R2(x) on the second, erfc = e^{-x^2} (1/sqrt(pi) - R3(1/x^2)
// / x^2) / x on the third; the complement is 1 - the other.  ex2 = e^{-x^2}
// is passed in: the pair force needs it anyway, so no second exponential is
// taken (its rounding, x^2 <= 16 here, stays below 2e-15 relative).
// Relative error below 4e-15 against the C library on [0, 6]
// (test_fp64_pair_energy_matches_erfc).
//
// The first two intervals share one Horner chain of eight steps whose
// coefficients each lane selects by its interval: R1's shorter numerator and
// denominator are padded with leading zero coefficients (the chain stays at
// exactly 0 until R1's first coefficient enters, so R1 is evaluated in its own
// order), and the final factor is x on the first interval, e^{-x^2} on the
// second.  A warp whose pairs straddle x = 0.46875 (a water molecule's own
// O-H and H-H pairs beside the others) then evaluates one rational function
// instead of both; selecting a coefficient is integer work, off the FP64 pipe.
__device__ __forceinline__ double erf_cody(double x, double ex2, bool want_erf)
{
    if (x > 4.0) {
        const double y = 1.0 / (x * x);
        double num = 1.63153871373020978e-2 * y, den = y;
        num = (num + 3.05326634961232344e-1) * y; den = (den + 2.56852019228982242e00) * y;
        num = (num + 3.60344899949804439e-1) * y; den = (den + 1.87295284992346725e00) * y;
        num = (num + 1.25781726111229246e-1) * y; den = (den + 5.27905102951428412e-1) * y;
        num = (num + 1.60837851487422766e-2) * y; den = (den + 6.05183413124413191e-2) * y;
        const double t = y * (num + 6.58749161529837803e-4) / (den + 2.33520497626869185e-3);
        const double r = ex2 * (0.56418958354775628695 - t) / x;
        return want_erf ? 1.0 - r : r;
    }
    const bool lo = x <= 0.46875;
    const double v = lo ? x * x : x;
    // numerator: R2's nine coefficients; R1's five after four zeros
    double num = (lo ? 0.0 : 2.15311535474403846e-8) * v;
    num = (num + (lo ? 0.0 : 5.64188496988670089e-1)) * v;
    num = (num + (lo ? 0.0 : 8.88314979438837594e00)) * v;
    num = (num + (lo ? 0.0 : 6.61191906371416295e01)) * v;
    num = (num + (lo ? 1.85777706184603153e-1 : 2.98635138197400131e02)) * v;
    num = (num + (lo ? 3.16112374387056560e00 : 8.81952221241769090e02)) * v;
    num = (num + (lo ? 1.13864154151050156e02 : 1.71204761263407058e03)) * v;
    num = (num + (lo ? 3.77485237685302021e02 : 2.05107837782607147e03)) * v;
    num += lo ? 3.20937758913846947e03 : 1.23033935479799725e03;
    // denominator: monic, R2's eight further coefficients; R1's four after zeros
    double den = (lo ? 0.0 : 1.0) * v;
    den = (den + (lo ? 0.0 : 1.57449261107098347e01)) * v;
    den = (den + (lo ? 0.0 : 1.17693950891312499e02)) * v;
    den = (den + (lo ? 0.0 : 5.37181101862009858e02)) * v;
    den = (den + (lo ? 1.0 : 1.62138957456669019e03)) * v;
    den = (den + (lo ? 2.36012909523441209e01 : 3.29079923573345963e03)) * v;
    den = (den + (lo ? 2.44024637934444173e02 : 4.36261909014324716e03)) * v;
    den = (den + (lo ? 1.28261652607737228e03 : 3.43936767414372164e03)) * v;
    den += lo ? 2.84423683343917062e03 : 1.23033935480374942e03;
    // erf = x R1 on the first interval, erfc = e^{-x^2} R2 on the second
    const double q = (lo ? x : ex2) * num / den;
    return lo == want_erf ? q : 1.0 - q;
}

// Minimum-image shift (-L, 0 or +L) of the FP64 coordinate difference
// x_j - x_i of two wrapped positions less than L/2 apart along that axis
// (every list member: r <= r_s <= L/2), from their 32-bit fixed-point codes:
// the plain difference crosses half the box exactly when the code difference
// wrapped to 32 bits has the opposite sign.  Adding the shift rounds once, as
// x - L rint(x / L) does, so the difference is the same double; the decision
// takes integer compares and selects instead of an FP64 multiply and round.
__device__ __forceinline__ double image_shift(uint32_t cj, uint32_t ci, double L)
{
    const int w = (int)(cj - ci);
    return (cj > ci && w < 0) ? -L : ((cj < ci && w > 0) ? L : 0.0);
}

// Position of the r-th set bit (r counted from 0) of m, r < popc(m): a
// binary search on the population counts of halves.
__device__ __forceinline__ int nth_set_bit(unsigned m, int r)
{
    int base = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (r >= c) {
            r -= c;
            m >>= w;
            base += w;
        }
    }
    return base;
}

// Floyd's algorithm over the ordinals [0, N_S), one slot per lane (p <= 32):
// slot k draws t_k uniform in [0, N_S - p + k] and inserts t_k, or N_S - p + k
// if t_k is already in the set.  Slot k's draw is in the set of slots 0..k-1
// exactly when an earlier slot drew the same value (that value is in the set
// whether or not that slot was replaced) or when t_k = N_S - p + m for an
// earlier slot m that was replaced.  The first test is one match over the
// warp; the second only chains through replaced slots of smaller index, so
// iterating it from the first test's result reaches the sequential
// algorithm's answer in at most p rounds (one round when no draw falls among
// the top p ordinals).  Returns lane k's inserted ordinal (lanes >= p: -1).
__device__ __forceinline__ int floyd_slot(const uint64_t* wa, int nshell, int p, int lane, unsigned lt_mask)
{
    const unsigned FULL = 0xffffffffu;
    const uint32_t jk = (uint32_t)(nshell - p + lane);
    const int tk = lane < p ? (int)uniform_below(wa[lane], jk + 1u) : -1 - lane;
    const bool d1 = (__match_any_sync(FULL, tk) & lt_mask) != 0u;
    const int m = tk - (nshell - p);
    const bool link = lane < p && m >= 0 && m < lane;
    unsigned dup = __ballot_sync(FULL, d1);
    if (__any_sync(FULL, link)) {
        for (int it = 0; it < p; ++it) {
            const unsigned nd = __ballot_sync(FULL, d1 || (link && ((dup >> (link ? m : 0)) & 1u)));
            if (nd == dup) break;
            dup = nd;
        }
    }
    return lane < p ? (((dup >> lane) & 1u) ? (int)jk : tk) : -1;
}

// floyd_slot for two atoms at once (their latency chains overlap): A's
// slots from waA over [0, nA), B's from waB over [0, nB); both nA, nB > p.
__device__ __forceinline__ void floyd_slot2(const uint64_t* waA, int nA, const uint64_t* waB, int nB, int p, int lane,
                                            unsigned lt_mask, int& selA, int& selB)
{
    const unsigned FULL = 0xffffffffu;
    const uint32_t jA = (uint32_t)(nA - p + lane), jB = (uint32_t)(nB - p + lane);
    const int tA = lane < p ? (int)uniform_below(waA[lane], jA + 1u) : -1 - lane;
    const int tB = lane < p ? (int)uniform_below(waB[lane], jB + 1u) : -1 - lane;
    const bool dA = (__match_any_sync(FULL, tA) & lt_mask) != 0u;
    const bool dB = (__match_any_sync(FULL, tB) & lt_mask) != 0u;
    const int mA = tA - (nA - p), mB = tB - (nB - p);
    const bool lA = lane < p && mA >= 0 && mA < lane, lB = lane < p && mB >= 0 && mB < lane;
    unsigned dupA = __ballot_sync(FULL, dA), dupB = __ballot_sync(FULL, dB);
    if (__any_sync(FULL, lA || lB)) {
        for (int it = 0; it < p; ++it) {
            const unsigned nA2 = __ballot_sync(FULL, dA || (lA && ((dupA >> (lA ? mA : 0)) & 1u)));
            const unsigned nB2 = __ballot_sync(FULL, dB || (lB && ((dupB >> (lB ? mB : 0)) & 1u)));
            if (nA2 == dupA && nB2 == dupB) break;
            dupA = nA2;
            dupB = nB2;
        }
    }
    selA = lane < p ? (((dupA >> lane) & 1u) ? (int)jA : tA) : -1;
    selB = lane < p ? (((dupB >> lane) & 1u) ? (int)jB : tB) : -1;
}

// Classification of one canonical segment [beg, end) of the source array:
// FP32 distance with exact integer decision inside the rounding bands.
template <bool SMALL>
__device__ __forceinline__ void dist_class(const float4 pj, bool valid, float xie, float yie, float zie,
                                           const RblGeom& g, float Lf, float invLf, bool& is_core, bool& is_shell,
                                           bool& amb)
{
    float dx = pj.x - xie, dy = pj.y - yie, dz = pj.z - zie;
    if (SMALL) {
        dx -= Lf * rintf(dx * invLf);
        dy -= Lf * rintf(dy * invLf);
        dz -= Lf * rintf(dz * invLf);
    }
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (!valid) r2 = 3.0e38f;
    // sorted FP32 thresholds tiny2 < rc2_lo <= rc2_hi < rs2_lo <= rs2_hi,
    // rounded outward on the host: (tiny2, rc2_lo) definite core,
    // (rc2_hi, rs2_lo) definite shell, above rs2_hi out; the rest is decided
    // exactly.  All decisions compare the same r2, so they partition exactly.
    is_core = r2 > g.tiny2 && r2 < g.rc2_lo;
    is_shell = r2 > g.rc2_hi && r2 < g.rs2_lo;
    amb = !is_core && !is_shell && r2 <= g.rs2_hi;
}

// Classification of one canonical segment [beg, end) of the source array:
// FP32 distance with exact integer decision inside the rounding bands.  Two
// chunks of 32 candidates are processed per iteration (their loads and
// arithmetic are independent) and appended in order; a tail of at most 32
// candidates takes a one-chunk iteration.
template <bool SMALL>
__device__ __forceinline__ void classify(const float4* __restrict__ src, int beg, int end, int goff, float xie,
                                         float yie, float zie, const RblArgs& a, int i, uint4 si, int lane,
                                         unsigned lt_mask, int* core_buf, int* shell_buf, int& ncore, int& nshell,
                                         bool& overlap, float Lf, float invLf)
{
    const RblGeom& g = a.g;
    const unsigned FULL = 0xffffffffu;
    int bb = beg;
    for (; end - bb > 32; bb += 64) {
        const int sa = bb + lane, sb = bb + 32 + lane;
        const bool vb = sb < end;
        const float4 pa = src[sa];
        const float4 pb = src[vb ? sb : beg];
        bool ca, sha, ma, cb, shb, mb;
        dist_class<SMALL>(pa, true, xie, yie, zie, g, Lf, invLf, ca, sha, ma);
        dist_class<SMALL>(pb, vb, xie, yie, zie, g, Lf, invLf, cb, shb, mb);
        const int ga = sa + goff, gb = sb + goff;
        if (__any_sync(FULL, ma || mb)) {
            if (ma) {
                unsigned long long d2 = d2_exact(si, a.s4[ga]);
                bool other = ga != i;
                ca = other && d2 <= a.c.Rc2;
                sha = other && d2 > a.c.Rc2 && d2 <= a.c.Rs2;
                overlap |= other && d2 == 0ull;
            }
            if (mb) {
                unsigned long long d2 = d2_exact(si, a.s4[gb]);
                bool other = gb != i;
                cb = other && d2 <= a.c.Rc2;
                shb = other && d2 > a.c.Rc2 && d2 <= a.c.Rs2;
                overlap |= other && d2 == 0ull;
            }
        }
        const unsigned cma = __ballot_sync(FULL, ca), sma = __ballot_sync(FULL, sha);
        const unsigned cmb = __ballot_sync(FULL, cb), smb = __ballot_sync(FULL, shb);
        const int nca = __popc(cma), nsa = __popc(sma);
        const int cpa = ncore + __popc(cma & lt_mask), spa = nshell + __popc(sma & lt_mask);
        const int cpb = ncore + nca + __popc(cmb & lt_mask), spb = nshell + nsa + __popc(smb & lt_mask);
        if (ca && cpa < a.core_cap) core_buf[cpa] = ga;
        if (sha && spa < a.shell_cap) shell_buf[spa] = ga;
        if (cb && cpb < a.core_cap) core_buf[cpb] = gb;
        if (shb && spb < a.shell_cap) shell_buf[spb] = gb;
        ncore += nca + __popc(cmb);
        nshell += nsa + __popc(smb);
    }
    if (bb < end) {
        const int sa = bb + lane;
        const bool va = sa < end;
        const float4 pa = src[va ? sa : beg];
        bool ca, sha, ma;
        dist_class<SMALL>(pa, va, xie, yie, zie, g, Lf, invLf, ca, sha, ma);
        const int ga = sa + goff;
        if (__any_sync(FULL, ma)) {
            if (ma) {
                unsigned long long d2 = d2_exact(si, a.s4[ga]);
                bool other = ga != i;
                ca = other && d2 <= a.c.Rc2;
                sha = other && d2 > a.c.Rc2 && d2 <= a.c.Rs2;
                overlap |= other && d2 == 0ull;
            }
        }
        const unsigned cma = __ballot_sync(FULL, ca), sma = __ballot_sync(FULL, sha);
        const int cpa = ncore + __popc(cma & lt_mask), spa = nshell + __popc(sma & lt_mask);
        if (ca && cpa < a.core_cap) core_buf[cpa] = ga;
        if (sha && spa < a.shell_cap) shell_buf[spa] = ga;
        ncore += __popc(cma);
        nshell += __popc(sma);
    }
}

// Exact decision of one candidate inside the rounding bands of its FP32
// distance (same rules as the stencil walk).
__device__ __forceinline__ void exact_class(const RblArgs& a, int i, uint4 si, int gj, bool& is_core, bool& is_shell,
                                            bool& overlap)
{
    const unsigned long long d2 = d2_exact(si, a.s4[gj]);
    const bool other = gj != i;
    is_core = other && d2 <= a.c.Rc2;
    is_shell = other && d2 > a.c.Rc2 && d2 <= a.c.Rs2;
    overlap |= other && d2 == 0ull;
}

// Classification of the concatenated candidate ranges of one pass of stencil
// rows, virtual positions [0, T).  Range k of the warp's table holds (staged
// index - position, global index - position); bit v of the start bitmap is
// set where a range begins.  Lane l of a 32-wide chunk takes position
// v = v0 + l (v0 a multiple of 32) and its range index is the number of range
// starts at or below v, less one: the starts below v0 are counted as the
// chunks go, the rest from the chunk's bitmap word, so every chunk but the
// last is full whatever the lengths of the ranges.  The staged positions
// carry their image shifts, so every candidate is compared with atom i's
// position (xi, yi, zi).  Four chunks per iteration (then two, then one),
// appended in order, as in the per-range walk.
__device__ __forceinline__ void classify_packed(const float4* __restrict__ stage, const int2* __restrict__ ranges,
                                                const unsigned* __restrict__ rstart, int T, float xi, float yi,
                                                float zi, const RblArgs& a, int i, uint4 si, int lane,
                                                unsigned lt_mask, int* core_buf, int* shell_buf, int& ncore,
                                                int& nshell, bool& overlap)
{
    const RblGeom& g = a.g;
    const unsigned FULL = 0xffffffffu;
    const unsigned le_mask = lt_mask | (1u << lane);
    int before = 0;                       // range starts below v0
    int v0 = 0;
    // four chunks per iteration while at least three are full: their loads,
    // distances and exact checks are independent (more work in flight per
    // warp against the fixed-latency dependencies); appended in chunk order
    for (; T - v0 > 96; v0 += 128) {
        unsigned w[4];
        int2 r[4];
        float4 pp[4];
        bool cc[4], ss[4], mm[4];
        int gg[4];
        int bc = before;
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = rstart[(v0 >> 5) + c];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            r[c] = ranges[bc + __popc(w[c] & le_mask) - 1];
            bc += __popc(w[c]);
        }
        before = bc;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int v = v0 + 32 * c + lane;
            const bool ok = c < 3 || v < T;
            pp[c] = stage[ok ? v + r[c].x : v0 + lane + r[0].x];
            gg[c] = v + r[c].y;
        }
        bool any_m = false;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool ok = c < 3 || (v0 + 96 + lane) < T;
            dist_class<false>(pp[c], ok, xi, yi, zi, g, 0.f, 0.f, cc[c], ss[c], mm[c]);
            mm[c] = mm[c] && gg[c] != i;        // i's own entry (r = 0) is no member: no exact test
            any_m |= mm[c];
        }
        if (__any_sync(FULL, any_m)) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (mm[c]) exact_class(a, i, si, gg[c], cc[c], ss[c], overlap);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const unsigned cm = __ballot_sync(FULL, cc[c]), sm = __ballot_sync(FULL, ss[c]);
            const int cp = ncore + __popc(cm & lt_mask), sp = nshell + __popc(sm & lt_mask);
            if (cc[c] && cp < a.core_cap) core_buf[cp] = gg[c];
            if (ss[c] && sp < a.shell_cap) shell_buf[sp] = gg[c];
            ncore += __popc(cm);
            nshell += __popc(sm);
        }
    }
    for (; T - v0 > 32; v0 += 64) {
        const unsigned wa = rstart[v0 >> 5], wb = rstart[(v0 >> 5) + 1];
        const int na = __popc(wa);
        const int2 ra = ranges[before + __popc(wa & le_mask) - 1];
        const int2 rb = ranges[before + na + __popc(wb & le_mask) - 1];
        before += na + __popc(wb);
        const int va = v0 + lane, vb = va + 32;
        const bool vbok = vb < T;
        const float4 pa = stage[va + ra.x];
        const float4 pb = stage[vbok ? vb + rb.x : va + ra.x];
        bool ca, sha, ma, cb, shb, mb;
        dist_class<false>(pa, true, xi, yi, zi, g, 0.f, 0.f, ca, sha, ma);
        dist_class<false>(pb, vbok, xi, yi, zi, g, 0.f, 0.f, cb, shb, mb);
        const int ga = va + ra.y, gb = vb + rb.y;
        ma = ma && ga != i;
        mb = mb && gb != i;
        if (__any_sync(FULL, ma || mb)) {
            if (ma) exact_class(a, i, si, ga, ca, sha, overlap);
            if (mb) exact_class(a, i, si, gb, cb, shb, overlap);
        }
        const unsigned cma = __ballot_sync(FULL, ca), sma = __ballot_sync(FULL, sha);
        const unsigned cmb = __ballot_sync(FULL, cb), smb = __ballot_sync(FULL, shb);
        const int nca = __popc(cma), nsa = __popc(sma);
        const int cpa = ncore + __popc(cma & lt_mask), spa = nshell + __popc(sma & lt_mask);
        const int cpb = ncore + nca + __popc(cmb & lt_mask), spb = nshell + nsa + __popc(smb & lt_mask);
        if (ca && cpa < a.core_cap) core_buf[cpa] = ga;
        if (sha && spa < a.shell_cap) shell_buf[spa] = ga;
        if (cb && cpb < a.core_cap) core_buf[cpb] = gb;
        if (shb && spb < a.shell_cap) shell_buf[spb] = gb;
        ncore += nca + __popc(cmb);
        nshell += nsa + __popc(smb);
    }
    if (v0 < T) {
        const unsigned wa = rstart[v0 >> 5];
        const int2 ra = ranges[before + __popc(wa & le_mask) - 1];
        const int va = v0 + lane;
        const bool vaok = va < T;
        const float4 pa = stage[vaok ? va + ra.x : 0];      // lanes past T: any staged slot, not classified
        bool ca, sha, ma;
        dist_class<false>(pa, vaok, xi, yi, zi, g, 0.f, 0.f, ca, sha, ma);
        const int ga = va + ra.y;
        ma = ma && ga != i;
        if (__any_sync(FULL, ma)) {
            if (ma) exact_class(a, i, si, ga, ca, sha, overlap);
        }
        const unsigned cma = __ballot_sync(FULL, ca), sma = __ballot_sync(FULL, sha);
        const int cpa = ncore + __popc(cma & lt_mask), spa = nshell + __popc(sma & lt_mask);
        if (ca && cpa < a.core_cap) core_buf[cpa] = ga;
        if (sha && spa < a.shell_cap) shell_buf[spa] = ga;
        ncore += __popc(cma);
        nshell += __popc(sma);
    }
}

// Classification of the concatenated candidate ranges of one pass against two
// atoms A and B of the same cell row at once (the ranges cover the union of
// their stencils).  The range lookup and the staged load of each candidate
// are shared; each atom gets its own FP32 distance and exact decision in the
// rounding bands.  Core members are appended in order to each atom's buffer;
// the shell membership of chunk k (positions 32k .. 32k+31) is kept as one
// ballot word per atom, smask[2k] for A and smask[2k+1] for B, so that shell
// ordinals can later be mapped back to candidates without a shell list.
// Without B (hasB false) B's sets are empty.  Two chunks per iteration, then
// one; lanes past T load a fixed staged slot and are not classified.
__device__ __forceinline__ void classify_pair(const float4* __restrict__ stage, const int2* __restrict__ ranges,
                                              const unsigned* __restrict__ rstart, int T, float4 pA, float4 pB,
                                              bool hasB, const RblArgs& a, int iA, int iB, uint4 sA, uint4 sB,
                                              int lane, unsigned lt_mask, int* coreA, int* coreB,
                                              unsigned* smask, int& ncA, int& ncB, bool& overlap)
{
    const RblGeom& g = a.g;
    const unsigned FULL = 0xffffffffu;
    const unsigned le_mask = lt_mask | (1u << lane);
    int before = 0;
    int v0 = 0;
    for (; T - v0 > 32; v0 += 64) {
        const unsigned wa = rstart[v0 >> 5], wb = rstart[(v0 >> 5) + 1];
        const int2 ra = ranges[before + __popc(wa & le_mask) - 1];
        const int2 rb = ranges[before + __popc(wa) + __popc(wb & le_mask) - 1];
        before += __popc(wa) + __popc(wb);
        const int va = v0 + lane, vb = va + 32;
        const bool vbok = vb < T;
        const float4 qa = stage[va + ra.x];
        const float4 qb = stage[vbok ? vb + rb.x : va + ra.x];
        const int ga = va + ra.y, gb = vb + rb.y;
        bool caA, saA, maA, cbA, sbA, mbA, caB, saB, maB, cbB, sbB, mbB;
        dist_class<false>(qa, true, pA.x, pA.y, pA.z, g, 0.f, 0.f, caA, saA, maA);
        dist_class<false>(qb, vbok, pA.x, pA.y, pA.z, g, 0.f, 0.f, cbA, sbA, mbA);
        dist_class<false>(qa, hasB, pB.x, pB.y, pB.z, g, 0.f, 0.f, caB, saB, maB);
        dist_class<false>(qb, hasB && vbok, pB.x, pB.y, pB.z, g, 0.f, 0.f, cbB, sbB, mbB);
        // an atom's own entry (r = 0) is no member: excluded by index, which
        // keeps it out of the exact test (one global load per atom saved)
        maA = maA && ga != iA;
        mbA = mbA && gb != iA;
        maB = maB && ga != iB;
        mbB = mbB && gb != iB;
        if (__any_sync(FULL, maA || mbA || maB || mbB)) {
            if (maA) exact_class(a, iA, sA, ga, caA, saA, overlap);
            if (mbA) exact_class(a, iA, sA, gb, cbA, sbA, overlap);
            if (maB) exact_class(a, iB, sB, ga, caB, saB, overlap);
            if (mbB) exact_class(a, iB, sB, gb, cbB, sbB, overlap);
        }
        const unsigned cma = __ballot_sync(FULL, caA), cmb = __ballot_sync(FULL, cbA);
        const unsigned cna = __ballot_sync(FULL, caB), cnb = __ballot_sync(FULL, cbB);
        const unsigned sma = __ballot_sync(FULL, saA), smb = __ballot_sync(FULL, sbA);
        const unsigned sna = __ballot_sync(FULL, saB), snb = __ballot_sync(FULL, sbB);
        const int pa = ncA + __popc(cma & lt_mask), pb = ncA + __popc(cma) + __popc(cmb & lt_mask);
        const int qa2 = ncB + __popc(cna & lt_mask), qb2 = ncB + __popc(cna) + __popc(cnb & lt_mask);
        if (caA && pa < a.core_cap) coreA[pa] = ga;
        if (cbA && pb < a.core_cap) coreA[pb] = gb;
        if (caB && qa2 < a.core_cap) coreB[qa2] = ga;
        if (cbB && qb2 < a.core_cap) coreB[qb2] = gb;
        ncA += __popc(cma) + __popc(cmb);
        ncB += __popc(cna) + __popc(cnb);
        if (lane == 0)
            reinterpret_cast<uint4*>(smask)[v0 >> 6] = make_uint4(sma, sna, smb, snb);
    }
    if (v0 < T) {
        const unsigned wa = rstart[v0 >> 5];
        const int2 ra = ranges[before + __popc(wa & le_mask) - 1];
        const int va = v0 + lane;
        const bool vaok = va < T;
        const float4 qa = stage[vaok ? va + ra.x : 0];
        const int ga = va + ra.y;
        bool caA, saA, maA, caB, saB, maB;
        dist_class<false>(qa, vaok, pA.x, pA.y, pA.z, g, 0.f, 0.f, caA, saA, maA);
        dist_class<false>(qa, hasB && vaok, pB.x, pB.y, pB.z, g, 0.f, 0.f, caB, saB, maB);
        maA = maA && ga != iA;
        maB = maB && ga != iB;
        if (__any_sync(FULL, maA || maB)) {
            if (maA) exact_class(a, iA, sA, ga, caA, saA, overlap);
            if (maB) exact_class(a, iB, sB, ga, caB, saB, overlap);
        }
        const unsigned cma = __ballot_sync(FULL, caA), cna = __ballot_sync(FULL, caB);
        const unsigned sma = __ballot_sync(FULL, saA), sna = __ballot_sync(FULL, saB);
        const int pa = ncA + __popc(cma & lt_mask), qa2 = ncB + __popc(cna & lt_mask);
        if (caA && pa < a.core_cap) coreA[pa] = ga;
        if (caB && qa2 < a.core_cap) coreB[qa2] = ga;
        ncA += __popc(cma);
        ncB += __popc(cna);
        if (lane == 0) reinterpret_cast<uint2*>(smask)[v0 >> 5] = make_uint2(sma, sna);
    }
}

// Classification of entries [t0, t0 + RBL_LGROUP) of atom i's stored list
// V(i) (Verlet-skin variant; nv entries in all, those of this step in the
// shared buffer vb) at the current positions: the exact rule on the
// fixed-point codes (minimum image by the 32-bit wrap), members appended in
// the order of V(i) to the core and shell buffers.  The four chunks' position
// loads are in flight together; V(i) never holds i.
__device__ __forceinline__ void classify_stored(const RblArgs& a, int i, uint4 si, const int* vb, int t0, int nv,
                                                int lane, unsigned lt_mask, int* core_buf, int* shell_buf,
                                                int& ncore, int& nshell, bool& overlap)
{
    const unsigned FULL = 0xffffffffu;
    int j[4];
    bool ok[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        ok[c] = t0 + 32 * c + lane < nv;
        j[c] = ok[c] ? vb[32 * c + lane] : i;
    }
    uint4 sj[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sj[c] = a.s4[j[c]];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const unsigned long long d2 = d2_exact(si, sj[c]);
        const bool cc = ok[c] && d2 <= a.c.Rc2;
        const bool ss = ok[c] && d2 > a.c.Rc2 && d2 <= a.c.Rs2;
        overlap |= ok[c] && d2 == 0ull;
        const unsigned cm = __ballot_sync(FULL, cc), sm = __ballot_sync(FULL, ss);
        const int cp = ncore + __popc(cm & lt_mask), sp = nshell + __popc(sm & lt_mask);
        if (cc && cp < a.core_cap) core_buf[cp] = j[c];
        if (ss && sp < a.shell_cap) shell_buf[sp] = j[c];
        ncore += __popc(cm);
        nshell += __popc(sm);
    }
}

template <bool MIXED, bool SMALL, bool ADJ, int LMODE = RBL_STENCIL>
__device__ __forceinline__ void rbl_body(const RblArgs& a, int slot, int nslots)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const RbeConsts& c = a.c;
    const RblGeom& g = a.g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int nc = c.n_cell, R = c.reach;
    const int G = g.G;
    const int p = c.p;
    const int p_pad = (p + 3) & ~3;
    const int nbk = p_pad / 4;

    // ---- shared layout ------------------------------------------------------
    const int nt2 = c.ntypes * c.ntypes;
    // (the list build keeps no core list here: the same layout as the host's)
    const SmemLayout lay = smem_layout(g, nt2, p, LMODE == RBL_BUILD ? 0 : a.core_cap, a.shell_cap,
                                       LMODE == RBL_STORED);
    float4* stage = reinterpret_cast<float4*>(smem);                              // [cap_stage]
    RowInfo* rows = reinterpret_cast<RowInfo*>(smem + lay.rows);                   // [nrows]
    int* cellpos = reinterpret_cast<int*>(smem + lay.cellpos);                     // [nrows * cpr]
    int* cellabs = reinterpret_cast<int*>(smem + lay.cellabs);                     // [nrows * cpr]
    const int cpr = g.cells_per_row + 1;
    double* s_c12 = reinterpret_cast<double*>(smem + lay.lj);
    double* s_c6 = s_c12 + nt2;
    double* s_sh = s_c6 + nt2;
    double* s_eps = s_sh + nt2;             // adjoint: eps_ab, sigma_ab, d shift
    double* s_sig = s_eps + nt2;
    double* s_dsde = s_sig + nt2;
    double* s_dsds = s_dsde + nt2;
    double* s_rc2 = s_dsds + nt2;           // squared LJ cutoff per pair type
    double* s_glj = s_rc2 + nt2;            // adjoint: [4][nt2] block accumulators
    // mixed forces: FP32 copies of (c12, c6, shift, squared cutoff) per type
    // pair, one 16-byte entry each, held where the adjoint keeps eps_ab and
    // sigma_ab (one conversion per block, one shared load per pair)
    float4* f_lj = reinterpret_cast<float4*>(smem + up16(lay.lj + 3 * sizeof(double) * (size_t)nt2));
    int2* ranges = reinterpret_cast<int2*>(smem + lay.warps + lay.wbytes * wib);          // [RBL_MAX_RANGES]
    unsigned* rstart = reinterpret_cast<unsigned*>(ranges + RBL_MAX_RANGES);              // [RBL_MAX_PACKED / 32]
    uint64_t* words = reinterpret_cast<uint64_t*>(rstart + RBL_MAX_PACKED / 32);         // [ga][p_pad]
    int* core_buf = reinterpret_cast<int*>(words + (size_t)p_pad * lay.ga);
    int* const core_buf_w = core_buf;
    int* shell_buf = core_buf + (LMODE == RBL_BUILD ? 0 : a.core_cap);
    int* sel = shell_buf + a.shell_cap;
    __shared__ int s_unit_ok;
    // completion barrier of the staging copies (one phase per staged unit)
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_phase;        // parity of the barrier's current phase
    __shared__ int s_stage_total;       // staged atoms of the current unit
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar, 1u);
        s_phase = 0u;
    }
    __syncthreads();
    __shared__ double red[WARPS][RBE_NPART_RBL];

    for (int t = threadIdx.x; t < nt2; t += blockDim.x) {
        int ti = t / c.ntypes, tj = t % c.ntypes;
        s_c12[t] = a.lj->c12[ti * RBE_MAXT + tj];
        s_c6[t] = a.lj->c6[ti * RBE_MAXT + tj];
        s_sh[t] = a.lj->shift[ti * RBE_MAXT + tj];
        s_rc2[t] = a.lj->rc2[ti * RBE_MAXT + tj];
        if (MIXED && !ADJ) {
            f_lj[t] = make_float4((float)s_c12[t], (float)s_c6[t], (float)s_sh[t], (float)s_rc2[t]);
        }
        if (ADJ) {
            s_eps[t] = a.lj->eps[ti * RBE_MAXT + tj];
            s_sig[t] = a.lj->sig[ti * RBE_MAXT + tj];
            s_dsde[t] = a.lj->dshift_de[ti * RBE_MAXT + tj];
            s_dsds[t] = a.lj->dshift_ds[ti * RBE_MAXT + tj];
            for (int q = 0; q < 4; ++q) s_glj[q * nt2 + t] = 0.0;
        }
    }

    const int naxis = SMALL ? nc : 2 * R + 1;
    const int nrows = naxis * naxis;
    const float Lf = (float)c.L;
    const float invLf = (float)c.invL;
    const float ncf = (float)nc;

    double acc_e[3] = {0.0, 0.0, 0.0};
    double acc_w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double acc_f[3] = {0.0, 0.0, 0.0};
    float facc_e[3] = {0.f, 0.f, 0.f}, facc_w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, facc_f[3] = {0.f, 0.f, 0.f};
    int fl_count = 0;

    const int units_per_row = (nc + G - 1) / G;
    const long nunits = (long)nc * nc * units_per_row;

    // Eq. (2.10) in FP32 (mixed path) for atom i (fixed-point si, kqi = k_e
    // q_i, (type, mol) ti) and partner j (sj, tj) with weight w: the Coulomb
    // factor erfc (erfc - 1 = -erf for a same-molecule pair, the Ewald
    // exclusion correction) and LJ; adds the force on i to ff and the
    // weighted energies and virial to the per-lane sums
    const float kef = (float)c.k_e, saf = (float)c.sqrt_alpha, tsaf = (float)c.two_sqrt_alpha_over_sqrt_pi;
    auto mixed_term = [&](const uint4 si, const float kqi, const int2 ti, const uint4 sj, const int2 tj, const float w,
                          float* ff) {
        const float dx = (float)(int)(sj.x - si.x) * c.Lfix;
        const float dy = (float)(int)(sj.y - si.y) * c.Lfix;
        const float dz = (float)(int)(sj.z - si.z) * c.Lfix;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float qq = kqi * __uint_as_float(sj.w);
        const float ar = saf * r;
        const float ex2 = __expf(-ar * ar);
        const float gauss = tsaf * ex2;
        const bool ex = ti.y == tj.y;
        const float ec = erfc_hastings(ar, ex2) - (ex ? 1.0f : 0.0f);
        const float ucoul = qq * ec * rinv;
        float sc = -qq * (ec * rinv + gauss) * rinv * rinv;
        const float4 lj = f_lj[ti.x * c.ntypes + tj.x];
        const bool nolj = ex || !(r2 < lj.w);
        const float c12 = nolj ? 0.f : lj.x, c6 = nolj ? 0.f : lj.y;
        const float ir2 = rinv * rinv;
        const float ir6 = ir2 * ir2 * ir2;
        sc -= (12.f * c12 * ir6 - 6.f * c6) * ir6 * ir2;
        const float ulj = (c12 * ir6 - c6) * ir6 - (nolj ? 0.f : lj.z);
        const float gx = w * sc * dx, gy = w * sc * dy, gz = w * sc * dz;
        ff[0] += gx; ff[1] += gy; ff[2] += gz;
        facc_e[0] += ex ? 0.f : w * ucoul;
        facc_e[1] += w * ulj;
        facc_e[2] += ex ? w * ucoul : 0.f;
        facc_w[0] += dx * gx; facc_w[1] += dy * gy; facc_w[2] += dz * gz;
        facc_w[3] += dx * gy; facc_w[4] += dx * gz; facc_w[5] += dy * gz;
    };
    // flush of the FP32 per-lane sums into FP64 every 16 atoms
    auto flush_sums = [&](int atoms) {
        fl_count += atoms;
        if (fl_count >= 16) {
#pragma unroll
            for (int q = 0; q < 3; ++q) { acc_e[q] += (double)facc_e[q]; facc_e[q] = 0.f; }
#pragma unroll
            for (int q = 0; q < 6; ++q) { acc_w[q] += (double)facc_w[q]; facc_w[q] = 0.f; }
#pragma unroll
            for (int q = 0; q < 3; ++q) { acc_f[q] += (double)facc_f[q]; facc_f[q] = 0.f; }
            fl_count = 0;
        }
    };

    // Two atoms per warp pass (mixed forward kernel, one pass of at most 32
    // stencil rows, staged units): the per-warp buffers are carved for A's and
    // B's core lists, the shell ballot words and their prefix counts, and the
    // materialised batches (see pair_two below)
    constexpr bool PAIRS = MIXED && !SMALL && !ADJ && LMODE == RBL_STENCIL;
    const bool pair_path = PAIRS && nrows <= 32 && lay.ga >= 2 && p <= 32 &&
                           a.shell_cap >= a.core_cap + RBL_PAIR_CARVE;

    // Per atom after its sets are known (core_buf[0 .. ncore), shell_buf[0 ..
    // nshell) in canonical order): the shell batch (Algorithm 1, shell step),
    // the pair terms of Eq. (2.10) and the debug record; wa_in holds the
    // atom's Philox words
    auto finish_atom = [&](const int i, const uint4 si, const int ncore, const int nshell, const bool overlap,
                           const uint64_t* wa_in) {
        if (__any_sync(FULL, overlap) && lane == 0) latch_status(a.status, RBE_ST_OVERLAP);
        if ((ncore > a.core_cap || nshell > a.shell_cap) && lane == 0) {
            latch_status(a.status, RBE_ST_CAPACITY);
            atomicMax(a.status + RBE_STW_NEED_CORE, ncore);      // what a retry needs
            atomicMax(a.status + RBE_STW_NEED_SHELL, nshell);
        }
        const int ncore_c = min(ncore, a.core_cap);
        const int gi = a.perm[i];

        // ---- 2. shell batch (Floyd over ordinals) -----------------------
        const bool sample = nshell > p;
        const int nb = sample ? p : nshell;
        const uint64_t* wa = wa_in;
        if (sample && c.shell_mode == 1) {
            // with replacement: slot k is ordinal floor(u_k N_S / 2^64)
            for (int k = lane; k < p; k += 32) sel[k] = (int)uniform_below(wa[k], (uint32_t)nshell);
        } else if (sample) {
            if (p <= 32) {
                // slot k on lane k
                const int mysel = floyd_slot(wa, nshell, p, lane, lt_mask);
                if (lane < p) sel[lane] = mysel;
            } else {
                for (int k = 0; k < p; ++k) {
                    const uint32_t jj = (uint32_t)(nshell - p + k);
                    const int t = (int)uniform_below(wa[k], jj + 1u);
                    bool dup = false;
                    for (int l = lane; l < k; l += 32) dup |= (sel[l] == t);
                    dup = __any_sync(FULL, dup);
                    if (lane == 0) sel[k] = dup ? (int)jj : t;
                    __syncwarp();
                }
            }
        }
        __syncwarp();

        // ---- 3. pair terms over C(i) and B(i) -----------------------------
        // Eq. (2.10) with the Coulomb factor erfc (erfc - 1 = -erf for a
        // same-molecule pair, the Ewald exclusion correction) and LJ.
        const int npairs = ncore_c + nb;
        const int2 ti = a.tm[i];
        if constexpr (ADJ) {
            // Gradients of E = 1/2 sum w_ij u_ij and of L = sum_i vt_i . F_real_i
            // (vt = v - mean v, which carries the momentum correction of
            // Eq. (2.13)) with respect to the charges and the LJ pair
            // parameters; the part of a pair that belongs to q_j is added
            // to atom j's slot atomically.
            const double vtx = a.vs[3 * (size_t)i] - a.vbar[0];
            const double vty = a.vs[3 * (size_t)i + 1] - a.vbar[1];
            const double vtz = a.vs[3 * (size_t)i + 2] - a.vbar[2];
            const double ke = c.k_e;
            const double4_32a pi = a.p4[i];
            double gE = 0.0, gL = 0.0;
            for (int t = lane; t < npairs; t += 32) {
                int j;
                double w;
                if (t < ncore_c) { j = core_buf[t]; w = 1.0; }
                else {
                    const int k = t - ncore_c;
                    const int ord = sample ? sel[k] : k;
                    j = shell_buf[min(ord, a.shell_cap - 1)];
                    w = sample ? (double)nshell / (double)p : 1.0;
                }
                const int2 tj = a.tm[j];
                const bool ex = ti.y == tj.y;
                double dx, dy, dz, qj, phi, h, r2;
                if (MIXED) {
                    const uint4 sj = a.s4[j];
                    const float fdx = (float)(int)(sj.x - si.x) * c.Lfix;
                    const float fdy = (float)(int)(sj.y - si.y) * c.Lfix;
                    const float fdz = (float)(int)(sj.z - si.z) * c.Lfix;
                    const float fr2 = fdx * fdx + fdy * fdy + fdz * fdz;
                    const float rinv = rsqrtf(fr2);
                    const float ar = (float)c.sqrt_alpha * fr2 * rinv;
                    const float gauss = (float)c.two_sqrt_alpha_over_sqrt_pi * __expf(-ar * ar);
                    const float ec = erfcf(ar) - (ex ? 1.0f : 0.0f);
                    phi = (double)(ec * rinv);
                    h = (double)(-(ec * rinv + gauss) * rinv * rinv);
                    dx = fdx; dy = fdy; dz = fdz; r2 = fr2;
                    qj = (double)__uint_as_float(sj.w);
                } else {
                    const double4_32a pj = a.p4[j];
                    const uint4 sj = a.s4[j];
                    dx = pj.x - pi.x + image_shift(sj.x, si.x, c.L);
                    dy = pj.y - pi.y + image_shift(sj.y, si.y, c.L);
                    dz = pj.z - pi.z + image_shift(sj.z, si.z, c.L);
                    r2 = dx * dx + dy * dy + dz * dz;
                    const double rinv = rsqrt(r2);     // one reciprocal square root, no division
                    const double rr = r2 * rinv;
                    const double ar = c.sqrt_alpha * rr;
                    const double ex2 = exp(-ar * ar);
                    const double gauss = c.two_sqrt_alpha_over_sqrt_pi * ex2;
                    const double ev = erf_cody(ar, ex2, ex), ec = ex ? -ev : ev;
                    phi = ec * rinv;
                    h = -(ec * rinv + gauss) * rinv * rinv;
                    qj = pj.w;
                }
                const double qi = MIXED ? (double)__uint_as_float(si.w) : pi.w;
                const double vd = vtx * dx + vty * dy + vtz * dz;
                gE += 0.5 * w * ke * qj * phi;
                gL += w * ke * qj * h * vd;
                atomicAdd(&a.gq_tr[2 * (size_t)j], 0.5 * w * ke * qi * phi);
                atomicAdd(&a.gq_tr[2 * (size_t)j + 1], w * ke * qi * h * vd);
                const int tt = ti.x * c.ntypes + tj.x;
                if (!ex && r2 < s_rc2[tt]) {
                    const double e = s_eps[tt], sg = s_sig[tt];
                    if (e != 0.0) {
                        const double ir2 = 1.0 / r2;
                        const double sr2 = sg * sg * ir2, sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
                        const double du_de = 4.0 * (sr12 - sr6) - s_dsde[tt];
                        const double du_ds = 4.0 * e * (12.0 * sr12 - 6.0 * sr6) / sg - s_dsds[tt];
                        const double dh_de = -(48.0 * sr12 - 24.0 * sr6) * ir2;
                        const double dh_ds = -e * (576.0 * sr12 - 144.0 * sr6) * ir2 / sg;
                        atomicAdd(&s_glj[0 * nt2 + tt], 0.5 * w * du_de);
                        atomicAdd(&s_glj[1 * nt2 + tt], 0.5 * w * du_ds);
                        atomicAdd(&s_glj[2 * nt2 + tt], w * dh_de * vd);
                        atomicAdd(&s_glj[3 * nt2 + tt], w * dh_ds * vd);
                    }
                }
            }
            gE = warp_sum(gE);
            gL = warp_sum(gL);
            if (lane == 0) {
                a.gq_own[2 * (size_t)i] = gE;
                a.gq_own[2 * (size_t)i + 1] = gL;
            }
        } else if (MIXED) {
            const float wsh = sample ? (float)nshell / (float)p : 1.0f;
            const float qi = __uint_as_float(si.w);
            float ff[3] = {0.f, 0.f, 0.f};
            auto pair_of = [&](int t, int& j, float& w) {
                if (t < ncore_c) { j = core_buf[t]; w = 1.0f; }
                else {
                    const int k = t - ncore_c;
                    const int ord = sample ? sel[k] : k;
                    j = shell_buf[min(ord, a.shell_cap - 1)];
                    w = wsh;
                }
            };
            const float kqi = kef * qi;
            auto term = [&](const uint4 sj, const int2 tj, const float w) { mixed_term(si, kqi, ti, sj, tj, w, ff); };
            // two pairs per lane per iteration (t, t + 32: the order of the
            // one-pair loop), their loads issued together
            for (int t = lane; t < npairs; t += 64) {
                const bool v2 = t + 32 < npairs;
                int j1, j2;
                float w1, w2;
                pair_of(t, j1, w1);
                if (v2) pair_of(t + 32, j2, w2);
                else { j2 = j1; w2 = 0.f; }
                const uint4 sj1 = a.s4[j1];
                const int2 tj1 = a.tm[j1];
                const uint4 sj2 = a.s4[j2];
                const int2 tj2 = a.tm[j2];
                term(sj1, tj1, w1);
                if (v2) term(sj2, tj2, w2);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) ff[q] = warp_sum(ff[q]);
            if (lane == 0) {
                float* Fr = reinterpret_cast<float*>(a.F_real);
                Fr[3 * (size_t)i + 0] = ff[0];
                Fr[3 * (size_t)i + 1] = ff[1];
                Fr[3 * (size_t)i + 2] = ff[2];
                facc_f[0] += ff[0]; facc_f[1] += ff[1]; facc_f[2] += ff[2];
            }
            flush_sums(1);
        } else {
            const double wsh = sample ? (double)nshell / (double)p : 1.0;
            const double4_32a pi = a.p4[i];
            double fi[3] = {0.0, 0.0, 0.0};
            for (int t = lane; t < npairs; t += 32) {
                int j;
                double w;
                if (t < ncore_c) { j = core_buf[t]; w = 1.0; }
                else {
                    const int k = t - ncore_c;
                    const int ord = sample ? sel[k] : k;
                    j = shell_buf[min(ord, a.shell_cap - 1)];
                    w = wsh;
                }
                const double4_32a pj = a.p4[j];
                const uint4 sj = a.s4[j];
                const int2 tj = a.tm[j];
                const double dx = pj.x - pi.x + image_shift(sj.x, si.x, c.L);
                const double dy = pj.y - pi.y + image_shift(sj.y, si.y, c.L);
                const double dz = pj.z - pi.z + image_shift(sj.z, si.z, c.L);
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double rinv = rsqrt(r2);         // one reciprocal square root, no division
                const double r = r2 * rinv;
                const double qq = c.k_e * pi.w * pj.w;
                const double ar = c.sqrt_alpha * r;
                const double ex2 = exp(-ar * ar);
                const double gauss = c.two_sqrt_alpha_over_sqrt_pi * ex2;
                const bool ex = ti.y == tj.y;
                // the exclusion term -erf is evaluated directly (not as
                // erfc - 1) to keep its full FP64 relative accuracy
                const double ev = erf_cody(ar, ex2, ex), ec = ex ? -ev : ev;
                const double ucoul = qq * ec * rinv;
                double s = -qq * (ec * rinv + gauss) * rinv * rinv;
                const int tt = ti.x * c.ntypes + tj.x;
                const bool nolj = ex || !(r2 < s_rc2[tt]);
                const double c12 = nolj ? 0.0 : s_c12[tt], c6 = nolj ? 0.0 : s_c6[tt];
                const double ir2 = rinv * rinv;
                const double ir6 = ir2 * ir2 * ir2;
                s -= (12.0 * c12 * ir6 - 6.0 * c6) * ir6 * ir2;
                const double ulj = (c12 * ir6 - c6) * ir6 - (nolj ? 0.0 : s_sh[tt]);
                const double gx = w * s * dx, gy = w * s * dy, gz = w * s * dz;
                fi[0] += gx; fi[1] += gy; fi[2] += gz;
                acc_e[0] += ex ? 0.0 : w * ucoul;
                acc_e[1] += w * ulj;
                acc_e[2] += ex ? w * ucoul : 0.0;
                acc_w[0] += dx * gx; acc_w[1] += dy * gy; acc_w[2] += dz * gz;
                acc_w[3] += dx * gy; acc_w[4] += dx * gz; acc_w[5] += dy * gz;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) fi[q] = warp_sum(fi[q]);
            if (lane == 0) {
                a.F_real[3 * (size_t)i + 0] = fi[0];
                a.F_real[3 * (size_t)i + 1] = fi[1];
                a.F_real[3 * (size_t)i + 2] = fi[2];
                acc_f[0] += fi[0]; acc_f[1] += fi[1]; acc_f[2] += fi[2];
            }
        }

        // ---- debug record (caller index order) ---------------------------
        if (a.debug) {
            if (lane == 0) { a.dbg_ncore[gi] = ncore; a.dbg_nshell[gi] = nshell; }
            for (int t = lane; t < a.dbg_cap; t += 32)
                a.dbg_core[(size_t)gi * a.dbg_cap + t] = t < ncore_c ? a.perm[core_buf[t]] : -1;
            for (int k = lane; k < p; k += 32) {
                int id = -1;
                if (k < nb) {
                    const int ord = sample ? sel[k] : k;
                    id = a.perm[shell_buf[min(ord, a.shell_cap - 1)]];
                }
                a.dbg_batch[(size_t)gi * p + k] = id;
            }
        }
        __syncwarp();
    };

    if constexpr (LMODE == RBL_STORED) {
        // atoms in sorted order, one per warp at a time, over the whole grid.
        // The entries of V(i) are classified RBL_LGROUP per step from a
        // per-warp double buffer in shared memory: while one step's entries
        // are classified, the next step's (the next group of V(i), or the
        // first of the warp's next atom) are being copied in, so the list read
        // from memory overlaps the position loads and the classification.
        int* lbuf = reinterpret_cast<int*>(smem + lay.warps + lay.wbytes * wib + lay.lbuf);
        const int stride = nslots * WARPS;
        // lane copies entries [t0 + 4 lane, t0 + 4 lane + 4) of V(ii) if the
        // first is below nvv (rows hold vcap entries, a multiple of 4, so
        // the copy stays in the row); one commit group per step
        auto issue = [&](int ii, int t0, int nvv, int buf) {
            const int e0 = t0 + 4 * lane;
            if (4 * lane < RBL_LGROUP && e0 < nvv)
                cp_async16(lbuf + buf * RBL_LGROUP + 4 * lane, a.vlist + (size_t)ii * a.vcap + e0);
            cp_async_commit();
        };
        int i = slot * WARPS + wib;
        int nv = i < a.n ? min(a.vcnt[i], a.vcap) : 0;
        int buf = 0;
        if (i < a.n) issue(i, 0, nv, buf);
        int kloc = 0;
        for (; i < a.n; i += stride, ++kloc) {
            const int inext = i + stride;
            const int nvn = inext < a.n ? min(a.vcnt[inext], a.vcap) : 0;
            const int aslot = kloc % lay.ga;
            if (aslot == 0) {
                __syncwarp();
                for (int t = lane; t < lay.ga * nbk; t += 32) {
                    const int aa = t / nbk, b = t - aa * nbk;
                    const int ii = i + stride * aa;
                    if (ii < a.n) {
                        uint64_t w[4];
                        philox4x64_10((uint64_t)a.perm[ii], (uint64_t)b, a.step, 1ull, c.seed, 0ull, w);
#pragma unroll
                        for (int qd = 0; qd < 4; ++qd) words[aa * p_pad + 4 * b + qd] = w[qd];
                    }
                }
                __syncwarp();
            }
            const uint4 si = a.s4[i];
            int ncore = 0, nshell = 0;
            bool overlap = false;
            const int ng = max(1, (nv + RBL_LGROUP - 1) / RBL_LGROUP);
            for (int gi = 0; gi < ng; ++gi) {
                if (gi + 1 < ng) issue(i, (gi + 1) * RBL_LGROUP, nv, buf ^ 1);
                else if (inext < a.n) issue(inext, 0, nvn, buf ^ 1);
                else cp_async_commit();                  // (an empty group)
                cp_async_wait<1>();                      // this step's copies have landed
                __syncwarp();
                classify_stored(a, i, si, lbuf + buf * RBL_LGROUP, gi * RBL_LGROUP, nv, lane, lt_mask, core_buf,
                                shell_buf, ncore, nshell, overlap);
                __syncwarp();                            // the buffer is refilled two steps on
                buf ^= 1;
            }
            finish_atom(i, si, ncore, nshell, overlap, words + (size_t)aslot * p_pad);
            nv = nvn;
        }
        cp_async_wait<0>();
    }
    for (long unit = LMODE == RBL_STORED ? nunits : slot; unit < nunits; unit += nslots) {
        const int ux = (int)(unit % units_per_row);
        const int uy = (int)((unit / units_per_row) % nc);
        const int uz = (int)(unit / ((long)units_per_row * nc));
        const int cx0 = ux * G;
        const int cx1 = min(cx0 + G, nc);           // exclusive
        const int rowbase_u = nc * (uy + nc * uz);
        const int A0 = a.cell_start[rowbase_u + cx0], A1 = a.cell_start[rowbase_u + cx1];
        if (A0 == A1) continue;                     // uniform across the block

        // ---- row table of the unit -------------------------------------------
        __syncthreads();
        const int ul = SMALL ? 0 : cx0 - R;
        const int uh = SMALL ? nc - 1 : cx1 - 1 + R;       // inclusive
        const int ncr = uh - ul + 1;                       // staged cells per row
        // (a) one thread per (row, cell): cell sizes; the row's descriptor
        for (int t = threadIdx.x; t < nrows * ncr; t += blockDim.x) {
            const int r = t / ncr, k = t - r * ncr;
            const int az = r / naxis, ay = r - az * naxis;
            const int zu = SMALL ? az : ring_row(az, uz, R, nc);
            const int yu = SMALL ? ay : ring_row(ay, uy, R, nc);
            const int zc = wrapc(zu, nc), yc = wrapc(yu, nc);
            const int rb = nc * (yc + nc * zc);
            const int w = wrapc(ul + k, nc);
            const int c0 = a.cell_start[rb + w];
            cellpos[r * cpr + k] = a.cell_start[rb + w + 1] - c0;
            cellabs[r * cpr + k] = c0;           // global start of the cell, for (d) and (e)
            if (k == 0) {
                RowInfo ri;
                ri.zc = zc;
                ri.yc = yc;
                ri.shz = SMALL ? 0.f : (zu < 0 ? -Lf : (zu >= nc ? Lf : 0.f));
                ri.shy = SMALL ? 0.f : (yu < 0 ? -Lf : (yu >= nc ? Lf : 0.f));
                ri.sbase = 0;
                ri.ul = ul;
                ri.goff[0] = ri.goff[1] = ri.goff[2] = 0;
                const int dz = zu - uz, dy = yu - uy;
                ri.zs = SMALL ? 0.f : (float)((dz > 0) - (dz < 0));
                ri.ys = SMALL ? 0.f : (float)((dy > 0) - (dy < 0));
                ri.zb = dz > 0 ? (float)(uz + dz) / ncf : (float)(uz + dz + 1) / ncf;
                ri.yb = dy > 0 ? (float)(uy + dy) / ncf : (float)(uy + dy + 1) / ncf;
                ri.pad = 0;
                rows[r] = ri;
            }
        }
        __syncthreads();
        // (b) exclusive prefix of the cell sizes of each row
        for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
            int* cp = cellpos + r * cpr;
            int acc = 0;
            for (int k = 0; k < ncr; ++k) {
                int v = cp[k];
                cp[k] = acc;
                acc += v;
            }
            cp[ncr] = acc;
        }
        __syncthreads();
        // (c) row bases in the staged array (warp 0 scans the row totals)
        if (wib == 0) {
            int carry = 0;
            for (int r0 = 0; r0 < nrows; r0 += 32) {
                const int r = r0 + lane;
                int v = r < nrows ? cellpos[r * cpr + ncr] : 0;
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += t;
                }
                if (r < nrows) rows[r].sbase = carry + incl - v;
                carry += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) {
                s_unit_ok = carry <= g.cap_stage;
                s_stage_total = carry;
            }
        }
        __syncthreads();
        const bool staged = s_unit_ok;
        if (a.debug && !staged && threadIdx.x == 0) atomicAdd(a.dbg_unstaged, 1);
        // (d) global - source offsets of the three pieces of each row
        for (int t = threadIdx.x; t < nrows * 3; t += blockDim.x) {
            const int r = t / 3, pc = t - 3 * r;
            const RowInfo& ri = rows[r];
            const int* cp = cellpos + r * cpr;
            const int ufirst = pc == 0 ? ul : (pc == 1 ? max(ul, 0) : max(ul, nc));
            int off = 0;
            if (staged && ufirst <= uh && (pc != 0 || ufirst < 0) && (pc != 1 || ufirst < nc))
                off = cellabs[r * cpr + (ufirst - ul)] - (ri.sbase + cp[ufirst - ul]);
            rows[r].goff[pc] = off;
        }
        // (e) stage the FP32 positions: one bulk asynchronous copy per
        // non-empty piece of a row (contiguous in the sorted arrays and in the
        // staged array), all completing on s_mbar, whose expected byte count
        // thread 0 posts; then each piece that lies across the box boundary
        // is moved in place to the periodic image adjacent to the unit (x: -L
        // below cell 0, +L past cell nc-1; y, z: the row's shift), so that
        // every staged candidate is compared with atom i's own position.  The
        // wait is bounded: a copy that never completes latches RBE_ST_STAGE
        // and the block stops.
        if (staged) {
            if (threadIdx.x == 0) mbar_arrive_expect_tx(&s_mbar, 16u * (uint32_t)s_stage_total);
            for (int t = threadIdx.x; t < nrows * 3; t += blockDim.x) {
                const int r = t / 3, pc = t - 3 * r;
                const int u0 = pc == 0 ? ul : (pc == 1 ? max(ul, 0) : max(ul, nc));
                const int u1 = pc == 0 ? min(uh, -1) : (pc == 1 ? min(uh, nc - 1) : uh);
                if (u0 > u1) continue;
                const int* cp = cellpos + r * cpr;
                const int len = cp[u1 - ul + 1] - cp[u0 - ul];
                if (len <= 0) continue;
                fence_proxy_async_smem();
                bulk_copy_g2s(stage + rows[r].sbase + cp[u0 - ul], a.f4 + cellabs[r * cpr + (u0 - ul)],
                              16u * (uint32_t)len, &s_mbar);
            }
            const uint32_t parity = s_phase;
            const bool done = mbar_wait_bounded(&s_mbar, parity, 1 << 22);
            if (__syncthreads_or(!done)) {
                if (threadIdx.x == 0) latch_status(a.status, RBE_ST_STAGE);
                mbar_wait_bounded(&s_mbar, parity, 1 << 22);     // copies still in flight
                return;
            }
            if (threadIdx.x == 0) s_phase = parity ^ 1u;     // read again after the unit's next barriers
            for (int r = wib; r < nrows; r += WARPS) {
                const int sb = rows[r].sbase;
                const float shy = rows[r].shy, shz = rows[r].shz;
                const int* cp = cellpos + r * cpr;
                for (int pc = 0; pc < 3; ++pc) {
                    const float shx = pc == 0 ? -Lf : (pc == 2 ? Lf : 0.f);
                    if (shx == 0.f && shy == 0.f && shz == 0.f) continue;
                    const int u0 = pc == 0 ? ul : (pc == 1 ? max(ul, 0) : max(ul, nc));
                    const int u1 = pc == 0 ? min(uh, -1) : (pc == 1 ? min(uh, nc - 1) : uh);
                    if (u0 > u1) continue;
                    const int len = cp[u1 - ul + 1] - cp[u0 - ul];
                    const int ss = sb + cp[u0 - ul];
                    for (int k = lane; k < len; k += 32) {
                        float4 q4 = stage[ss + k];
                        q4.x += shx;
                        q4.y += shy;
                        q4.z += shz;
                        stage[ss + k] = q4;
                    }
                }
            }
        }
        __syncthreads();

        // ---- atoms of the unit -------------------------------------------------
        // one_atom: lists, batch and pair terms of atom i, whose Philox words
        // are wa_in[0 .. p_pad)
        auto one_atom = [&](const int i, const uint64_t* wa_in) {
            int* core_buf = LMODE == RBL_BUILD ? a.vlist + (size_t)i * a.vcap : core_buf_w;
            const uint4 si = a.s4[i];
            const float4 fi4 = a.f4[i];
            const int cx = (int)cell_of_fixed(si.x, nc);
            const float fx = (float)si.x * 2.3283064365386963e-10f;
            const float fy = (float)si.y * 2.3283064365386963e-10f;
            const float fz = (float)si.z * 2.3283064365386963e-10f;
            int ncore = 0, nshell = 0;
            bool overlap = false;

            // ---- 1. classify the stencil in canonical order ------------------
            for (int rb0 = 0; rb0 < nrows; rb0 += 32) {
                // lane r describes row rb0 + r for this atom: up to two
                // canonical segments [b, e) of the source array
                int b1 = 0, e1 = 0, b2 = 0, e2 = 0, o1 = 0, o2 = 0;
                float x1 = 0.f, x2 = 0.f, yie = 0.f, zie = 0.f;
                const int r = rb0 + lane;
                if (r < nrows) {
                    const RowInfo& ri = rows[r];
                    const int* cp = cellpos + r * cpr;
                    // staged positions carry the row's image shift already
                    yie = staged ? fi4.y : fi4.y - ri.shy;
                    zie = staged ? fi4.z : fi4.z - ri.shz;
                    const int rbw = nc * (ri.yc + nc * ri.zc);
                    const int base = staged ? ri.sbase : 0;
                    if (SMALL) {
                        b1 = staged ? base : a.cell_start[rbw];
                        e1 = b1 + cp[nc];
                        o1 = ri.goff[1];
                        x1 = fi4.x;
                    } else {
                        const float gz = fmaxf(0.f, ri.zs * (ri.zb - fz));
                        const float gy = fmaxf(0.f, ri.ys * (ri.yb - fy));
                        const float g2 = gz * gz + gy * gy;
                        if (g2 <= c.rs_frac2) {
                            const float hx = sqrtf(c.rs_frac2 - g2) + 1e-5f;
                            const int dlo = max(-R, (int)floorf((fx - hx) * ncf) - cx);
                            const int dhi = min(R, (int)floorf((fx + hx) * ncf) - cx);
                            const int ua = cx + dlo, ub = cx + dhi;     // unwrapped, within [ul, uh]
                            // canonical order: ascending wrapped index
                            int lo1, hi1, lo2 = 1, hi2 = 0;
                            if (ua < 0) { lo1 = 0; hi1 = ub; lo2 = ua; hi2 = -1; }
                            else if (ub >= nc) { lo1 = nc; hi1 = ub; lo2 = ua; hi2 = nc - 1; }
                            else { lo1 = ua; hi1 = ub; }
                            const float H = hx * Lf;
                            const float4* srcp = staged ? stage : a.f4;
                            {
                                const int pc = lo1 >= nc ? 2 : 1;
                                if (staged) { b1 = base + cp[lo1 - ul]; e1 = base + cp[hi1 - ul + 1]; }
                                else { b1 = a.cell_start[rbw + wrapc(lo1, nc)]; e1 = b1 + cp[hi1 - ul + 1] - cp[lo1 - ul]; }
                                o1 = ri.goff[pc];
                                x1 = staged ? fi4.x : fi4.x - (pc == 2 ? Lf : 0.f);
                                trim_segment(srcp, b1, e1, cp[lo1 - ul + 1] - cp[lo1 - ul], cp[hi1 - ul + 1] - cp[hi1 - ul],
                                             lo1 == hi1, x1, H);
                            }
                            if (lo2 <= hi2) {
                                const int pc = lo2 < 0 ? 0 : 1;
                                if (staged) { b2 = base + cp[lo2 - ul]; e2 = base + cp[hi2 - ul + 1]; }
                                else { b2 = a.cell_start[rbw + wrapc(lo2, nc)]; e2 = b2 + cp[hi2 - ul + 1] - cp[lo2 - ul]; }
                                o2 = ri.goff[pc];
                                x2 = staged ? fi4.x : fi4.x - (pc == 0 ? -Lf : 0.f);
                                trim_segment(srcp, b2, e2, cp[lo2 - ul + 1] - cp[lo2 - ul], cp[hi2 - ul + 1] - cp[hi2 - ul],
                                             lo2 == hi2, x2, H);
                            }
                        }
                    }
                }
                if (!SMALL && staged) {
                    // concatenate the pass's segments in canonical order (row
                    // by row, each row's first segment before its second):
                    // one warp scan of (candidates, segments), packed in one
                    // word (both stay below 2^16: the segments are disjoint
                    // parts of the staged array), gives each lane the virtual
                    // position and table slot of its row's segments
                    const int n1 = e1 - b1, n2 = e2 - b2;
                    const int own = n1 + n2 + (((n1 > 0) + (n2 > 0)) << 16);
                    int incl = own;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += t;
                    }
                    const int T = __shfl_sync(FULL, incl, 31) & 0xffff;
                    if (a.debug && T > RBL_MAX_PACKED && lane == 0) atomicAdd(a.dbg_unstaged + 1, 1);
                    if (T <= RBL_MAX_PACKED) {
                        for (int w = lane; w < ((T + 31) >> 5); w += 32) rstart[w] = 0u;
                        __syncwarp();
                        int v = (incl - own) & 0xffff, k = (incl - own) >> 16;
                        if (n1 > 0) {
                            ranges[k++] = make_int2(b1 - v, b1 + o1 - v);
                            atomicOr(&rstart[v >> 5], 1u << (v & 31));
                            v += n1;
                        }
                        if (n2 > 0) {
                            ranges[k] = make_int2(b2 - v, b2 + o2 - v);
                            atomicOr(&rstart[v >> 5], 1u << (v & 31));
                        }
                        __syncwarp();
                        if (T > 0)
                            classify_packed(stage, ranges, rstart, T, fi4.x, fi4.y, fi4.z, a, i, si, lane, lt_mask,
                                            core_buf, shell_buf, ncore, nshell, overlap);
                        __syncwarp();        // the tables are rewritten by the next pass
                        continue;
                    }
                }
                // walk the non-empty segments in canonical order
                const unsigned m1 = __ballot_sync(FULL, e1 > b1), m2 = __ballot_sync(FULL, e2 > b2);
                unsigned mm = m1 | m2;
                while (mm) {
                    const int rr = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const float ry = __shfl_sync(FULL, yie, rr), rz = __shfl_sync(FULL, zie, rr);
                    if ((m1 >> rr) & 1u) {
                        const int beg = __shfl_sync(FULL, b1, rr), end = __shfl_sync(FULL, e1, rr);
                        const int go = __shfl_sync(FULL, o1, rr);
                        const float rx = __shfl_sync(FULL, x1, rr);
                        if (staged) classify<SMALL>(stage, beg, end, go, rx, ry, rz, a, i, si, lane, lt_mask, core_buf,
                                                    shell_buf, ncore, nshell, overlap, Lf, invLf);
                        else classify<SMALL>(a.f4, beg, end, go, rx, ry, rz, a, i, si, lane, lt_mask, core_buf,
                                             shell_buf, ncore, nshell, overlap, Lf, invLf);
                    }
                    if ((m2 >> rr) & 1u) {
                        const int beg = __shfl_sync(FULL, b2, rr), end = __shfl_sync(FULL, e2, rr);
                        const int go = __shfl_sync(FULL, o2, rr);
                        const float rx = __shfl_sync(FULL, x2, rr);
                        if (staged) classify<SMALL>(stage, beg, end, go, rx, ry, rz, a, i, si, lane, lt_mask, core_buf,
                                                    shell_buf, ncore, nshell, overlap, Lf, invLf);
                        else classify<SMALL>(a.f4, beg, end, go, rx, ry, rz, a, i, si, lane, lt_mask, core_buf,
                                             shell_buf, ncore, nshell, overlap, Lf, invLf);
                    }
                }
            }
            if constexpr (LMODE == RBL_BUILD) {
                // the stored list V(i): every member within r_s + skin (the
                // "core" of this launch's radii), canonical order, written
                // by the classification straight into the list
                if (__any_sync(FULL, overlap) && lane == 0) latch_status(a.status, RBE_ST_OVERLAP);
                if (ncore > a.vcap && lane == 0) {
                    latch_status(a.status, RBE_ST_CAPACITY);
                    atomicMax(a.status + RBE_STW_NEED_LIST, ncore);
                }
                if (lane == 0) a.vcnt[i] = min(ncore, a.vcap);
                __syncwarp();
            } else {
                finish_atom(i, si, ncore, nshell, overlap, wa_in);
            }
        };
        if (PAIRS && pair_path && staged) {
            // Atoms A = i and B = i + 1 of the unit per warp pass.  Their
            // stencils are the same 25 rows (one x-row of cells), so each
            // lane cuts its row to the hull of A's and B's x ranges, and the
            // concatenated candidates, in canonical order, are classified
            // against both (classify_pair).  A pass whose concatenation
            // exceeds RBL_MAX_PACKED falls back to one_atom for A and B.
            int* coreA = core_buf;
            int* coreB = shell_buf;
            unsigned* smask = reinterpret_cast<unsigned*>(shell_buf + a.core_cap);   // [2 * 64]
            int* pfxA = reinterpret_cast<int*>(smask + 128);                        // [64]
            int* pfxB = pfxA + 64;                                                   // [64]
            int* pfxR = pfxB + 64;                                                   // [64]
            int* jA = pfxR + 64;                                                     // [32]
            int* jB = jA + 32;                                                       // [32]
            int* selA = sel;
            int* selB = jB + 32;                                                     // [32]
            const int gp = lay.ga >> 1;       // pairs whose Philox words are made in one pass
            int kp = 0;
            for (int i = A0 + 2 * wib; i < A1; i += 2 * WARPS, ++kp) {
                const int pslot = kp % gp;
                if (pslot == 0) {
                    __syncwarp();
                    for (int t = lane; t < 2 * gp * nbk; t += 32) {
                        const int aa = t / nbk, b = t - aa * nbk;
                        const int ii = i + 2 * WARPS * (aa >> 1) + (aa & 1);
                        if (ii < A1) {
                            uint64_t w[4];
                            philox4x64_10((uint64_t)a.perm[ii], (uint64_t)b, a.step, 1ull, c.seed, 0ull, w);
#pragma unroll
                            for (int qd = 0; qd < 4; ++qd) words[aa * p_pad + 4 * b + qd] = w[qd];
                        }
                    }
                    __syncwarp();
                }
                const uint64_t* waA = words + (size_t)(2 * pslot) * p_pad;
                const uint64_t* waB = waA + p_pad;
                const bool hasB = i + 1 < A1;
                const int iA = i, iB = hasB ? i + 1 : i;
                const uint4 sA = a.s4[iA], sB = a.s4[iB];
                const float4 pA = a.f4[iA], pB = a.f4[iB];
                const int cxA = (int)cell_of_fixed(sA.x, nc), cxB = (int)cell_of_fixed(sB.x, nc);
                const float fxA = (float)sA.x * 2.3283064365386963e-10f, fxB = (float)sB.x * 2.3283064365386963e-10f;
                const float fyA = (float)sA.y * 2.3283064365386963e-10f, fyB = (float)sB.y * 2.3283064365386963e-10f;
                const float fzA = (float)sA.z * 2.3283064365386963e-10f, fzB = (float)sB.z * 2.3283064365386963e-10f;
                if (hasB && cxB - cxA + 2 * R + 1 > nc) {
                    // the hull of the two stencils would hold a cell twice
                    // (small boxes with empty cells between A and B)
                    one_atom(iA, waA);
                    one_atom(iB, waB);
                    continue;
                }

                // ---- 1. rows: segments of the hull of A's and B's x ranges -----
                int b1 = 0, e1 = 0, b2 = 0, e2 = 0, o1 = 0, o2 = 0;
                if (lane < nrows) {
                    const RowInfo& ri = rows[lane];
                    const int* cp = cellpos + lane * cpr;
                    const int base = ri.sbase;
                    const float gzA = fmaxf(0.f, ri.zs * (ri.zb - fzA)), gyA = fmaxf(0.f, ri.ys * (ri.yb - fyA));
                    const float gzB = fmaxf(0.f, ri.zs * (ri.zb - fzB)), gyB = fmaxf(0.f, ri.ys * (ri.yb - fyB));
                    const float g2A = gzA * gzA + gyA * gyA, g2B = gzB * gzB + gyB * gyB;
                    const bool okA = g2A <= c.rs_frac2, okB = hasB && g2B <= c.rs_frac2;
                    if (okA || okB) {
                        const float hxA = okA ? sqrtf(c.rs_frac2 - g2A) + 1e-5f : 0.f;
                        const float hxB = okB ? sqrtf(c.rs_frac2 - g2B) + 1e-5f : 0.f;
                        const float flo = okA ? (okB ? fminf(fxA - hxA, fxB - hxB) : fxA - hxA) : fxB - hxB;
                        const float fhi = okA ? (okB ? fmaxf(fxA + hxA, fxB + hxB) : fxA + hxA) : fxB + hxB;
                        const float xlo = okA ? (okB ? fminf(pA.x - hxA * Lf, pB.x - hxB * Lf) : pA.x - hxA * Lf)
                                              : pB.x - hxB * Lf;
                        const float xhi = okA ? (okB ? fmaxf(pA.x + hxA * Lf, pB.x + hxB * Lf) : pA.x + hxA * Lf)
                                              : pB.x + hxB * Lf;
                        // unwrapped cells of the hull, within A's and B's
                        // stencils (both inside the staged range [ul, uh])
                        const int ua = max(cxA - R, (int)floorf(flo * ncf));
                        const int ub = min(cxB + R, (int)floorf(fhi * ncf));
                        int lo1, hi1, lo2 = 1, hi2 = 0;
                        if (ua < 0) { lo1 = 0; hi1 = ub; lo2 = ua; hi2 = -1; }
                        else if (ub >= nc) { lo1 = nc; hi1 = ub; lo2 = ua; hi2 = nc - 1; }
                        else { lo1 = ua; hi1 = ub; }
                        b1 = base + cp[lo1 - ul];
                        e1 = base + cp[hi1 - ul + 1];
                        o1 = ri.goff[lo1 >= nc ? 2 : 1];
                        trim_range(stage, b1, e1, cp[lo1 - ul + 1] - cp[lo1 - ul], cp[hi1 - ul + 1] - cp[hi1 - ul],
                                   lo1 == hi1, xlo, xhi);
                        if (lo2 <= hi2) {
                            b2 = base + cp[lo2 - ul];
                            e2 = base + cp[hi2 - ul + 1];
                            o2 = ri.goff[lo2 < 0 ? 0 : 1];
                            trim_range(stage, b2, e2, cp[lo2 - ul + 1] - cp[lo2 - ul], cp[hi2 - ul + 1] - cp[hi2 - ul],
                                       lo2 == hi2, xlo, xhi);
                        }
                    }
                }
                // concatenation in canonical order (as in one_atom)
                const int n1 = e1 - b1, n2 = e2 - b2;
                const int own = n1 + n2 + (((n1 > 0) + (n2 > 0)) << 16);
                int incl = own;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += t;
                }
                const int T = __shfl_sync(FULL, incl, 31) & 0xffff;
                if (T >= RBL_MAX_PACKED) {
                    // (below 2048 candidates every prefix count fits the 11-bit
                    // fields packed below)
                    if (a.debug && lane == 0) atomicAdd(a.dbg_unstaged + 1, 1);
                    one_atom(iA, waA);
                    if (hasB) one_atom(iB, waB);
                    continue;
                }
                const int nch = (T + 31) >> 5;
                for (int w = lane; w < nch; w += 32) rstart[w] = 0u;
                __syncwarp();
                {
                    int v = (incl - own) & 0xffff, k = (incl - own) >> 16;
                    if (n1 > 0) {
                        ranges[k++] = make_int2(b1 - v, b1 + o1 - v);
                        atomicOr(&rstart[v >> 5], 1u << (v & 31));
                        v += n1;
                    }
                    if (n2 > 0) {
                        ranges[k] = make_int2(b2 - v, b2 + o2 - v);
                        atomicOr(&rstart[v >> 5], 1u << (v & 31));
                    }
                }
                __syncwarp();

                // ---- 2. classification against A and B -----------------------
                int ncA = 0, ncB = 0;
                bool overlap = false;
                if (T > 0)
                    classify_pair(stage, ranges, rstart, T, pA, pB, hasB, a, iA, iB, sA, sB, lane, lt_mask, coreA,
                                  coreB, smask, ncA, ncB, overlap);
                __syncwarp();
                if (__any_sync(FULL, overlap) && lane == 0) latch_status(a.status, RBE_ST_OVERLAP);
                if ((ncA > a.core_cap || ncB > a.core_cap) && lane == 0) {
                    latch_status(a.status, RBE_ST_CAPACITY);
                    atomicMax(a.status + RBE_STW_NEED_CORE, max(ncA, ncB));
                }
                const int ncAc = min(ncA, a.core_cap), ncBc = min(ncB, a.core_cap);
                // the first pair-term step of each half-warp (pairs l16 and
                // l16 + 16 of its atom: core members when the core holds 32 or
                // more) has its partner loads issued now, so that they land
                // while the batches are drawn and located
                const bool pre = (lane < 16 ? ncAc : ncBc) >= 32 && (lane < 16 || hasB);
                uint4 ps1 = make_uint4(0u, 0u, 0u, 0u), ps2 = ps1;
                int2 pt1 = make_int2(0, 0), pt2 = pt1;
                if (pre) {
                    const int* cX = lane < 16 ? coreA : coreB;
                    const int j1 = cX[lane & 15], j2 = cX[(lane & 15) + 16];
                    ps1 = a.s4[j1];
                    pt1 = a.tm[j1];
                    ps2 = a.s4[j2];
                    pt2 = a.tm[j2];
                }

                // exclusive prefix counts over the chunks (two per lane): shell
                // members of A and B, range starts
                int nsA, nsB;
                {
                    const unsigned wA0 = lane < nch ? smask[2 * lane] : 0u, wB0 = lane < nch ? smask[2 * lane + 1] : 0u;
                    const unsigned wA1 = lane + 32 < nch ? smask[2 * lane + 64] : 0u;
                    const unsigned wB1 = lane + 32 < nch ? smask[2 * lane + 65] : 0u;
                    const unsigned r0 = lane < nch ? rstart[lane] : 0u, r1 = lane + 32 < nch ? rstart[lane + 32] : 0u;
                    // three counts per word packed in one int: A | B << 11 | R << 22 (each < 2^11)
                    const int c0 = __popc(wA0) | (__popc(wB0) << 11) | (__popc(r0) << 22);
                    const int c1 = __popc(wA1) | (__popc(wB1) << 11) | (__popc(r1) << 22);
                    int s0 = c0, s1 = c1;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t0 = __shfl_up_sync(FULL, s0, o), t1 = __shfl_up_sync(FULL, s1, o);
                        if (lane >= o) { s0 += t0; s1 += t1; }
                    }
                    const int tot0 = __shfl_sync(FULL, s0, 31);
                    const int ex0 = s0 - c0, ex1 = tot0 + s1 - c1;
                    if (lane < nch) {
                        pfxA[lane] = ex0 & 0x7ff; pfxB[lane] = (ex0 >> 11) & 0x7ff; pfxR[lane] = ex0 >> 22;
                    }
                    if (lane + 32 < nch) {
                        pfxA[lane + 32] = ex1 & 0x7ff; pfxB[lane + 32] = (ex1 >> 11) & 0x7ff; pfxR[lane + 32] = ex1 >> 22;
                    }
                    const int all = tot0 + __shfl_sync(FULL, s1, 31);
                    nsA = all & 0x7ff;
                    nsB = hasB ? (all >> 11) & 0x7ff : 0;
                }
                __syncwarp();

                // ---- 3. batches: ordinals (Floyd), then the members they name --
                const bool sampA = nsA > p, sampB = nsB > p;
                auto draw = [&](int nshell, const uint64_t* wa, int* out) {
                    if (c.shell_mode == 1) {
                        if (lane < p) out[lane] = (int)uniform_below(wa[lane], (uint32_t)nshell);
                        return;
                    }
                    const int mysel = floyd_slot(wa, nshell, p, lane, lt_mask);
                    if (lane < p) out[lane] = mysel;
                };
                if (sampA && sampB && c.shell_mode != 1) {
                    int sa, sb;
                    floyd_slot2(waA, nsA, waB, nsB, p, lane, lt_mask, sa, sb);
                    if (lane < p) { selA[lane] = sa; selB[lane] = sb; }
                } else {
                    if (sampA) draw(nsA, waA, selA);
                    if (sampB) draw(nsB, waB, selB);
                }
                __syncwarp();
                // member of ordinal t of the shell: chunk c with pfx[c] <= t <
                // pfx[c + 1] (binary search), the (t - pfx[c])-th set bit of
                // its ballot word, then the range holding that position
                // (A's and B's searches interleaved: two independent chains)
                const int nbA = sampA ? p : nsA, nbB = sampB ? p : nsB;
                if (lane < nbA || lane < nbB) {
                    const bool doA = lane < nbA, doB = lane < nbB;
                    const int tA = doA ? (sampA ? selA[lane] : lane) : 0;
                    const int tB = doB ? (sampB ? selB[lane] : lane) : 0;
                    // (the two intervals can differ in length by one after
                    // the same number of halvings: each search stops on its own)
                    int loA = 0, hiA = nch, loB = 0, hiB = nch;
                    while (hiA - loA > 1 || hiB - loB > 1) {
                        const int mA = (loA + hiA) >> 1, mB = (loB + hiB) >> 1;
                        const int pa = pfxA[mA], pb = pfxB[mB];
                        if (hiA - loA > 1) {
                            if (pa <= tA) loA = mA;
                            else hiA = mA;
                        }
                        if (hiB - loB > 1) {
                            if (pb <= tB) loB = mB;
                            else hiB = mB;
                        }
                    }
                    const int bitA = nth_set_bit(smask[2 * loA], tA - pfxA[loA]);
                    const int bitB = nth_set_bit(smask[2 * loB + 1], tB - pfxB[loB]);
                    const unsigned uptoA = bitA == 31 ? 0xffffffffu : ((2u << bitA) - 1u);
                    const unsigned uptoB = bitB == 31 ? 0xffffffffu : ((2u << bitB) - 1u);
                    // (a lane without an ordinal for A or B searched for ordinal
                    // 0 there; its index is clamped and its result unused)
                    const int rA = max(pfxR[loA] + __popc(rstart[loA] & uptoA) - 1, 0);
                    const int rB = max(pfxR[loB] + __popc(rstart[loB] & uptoB) - 1, 0);
                    const int jA_ = 32 * loA + bitA + ranges[rA].y;
                    const int jB_ = 32 * loB + bitB + ranges[rB].y;
                    if (doA) jA[lane] = jA_;
                    if (doB) jB[lane] = jB_;
                }
                __syncwarp();

                // ---- 4. pair terms of A and B on the lanes of the warp ---------
                // lanes 0-15 take A's pairs, lanes 16-31 B's: each lane keeps
                // one atom, so the pair term needs no per-pair choice between
                // A and B; two pairs per lane per iteration (k, k + 16), their
                // loads issued together
                const int npA = ncAc + nbA, npB = hasB ? ncBc + nbB : 0;
                const bool hb = lane >= 16;
                const int l16 = lane & 15;
                const int npX = hb ? npB : npA, ncX = hb ? ncBc : ncAc;
                const float wshX = hb ? (sampB ? (float)nsB / (float)p : 1.0f) : (sampA ? (float)nsA / (float)p : 1.0f);
                const int* coreX = hb ? coreB : coreA;
                const int* jX = hb ? jB : jA;
                const uint4 sX = hb ? sB : sA;
                const int2 tiX = a.tm[hb ? iB : iA];
                const float kqX = kef * __uint_as_float(sX.w);
                float ff[3] = {0.f, 0.f, 0.f};
                auto pair_of = [&](int k, int& j, float& w) {
                    if (k < ncX) { j = coreX[k]; w = 1.0f; }
                    else { j = jX[k - ncX]; w = wshX; }
                };
                int k0 = l16;
                if (pre) {
                    mixed_term(sX, kqX, tiX, ps1, pt1, 1.0f, ff);
                    mixed_term(sX, kqX, tiX, ps2, pt2, 1.0f, ff);
                    k0 += 32;
                }
                for (int k = k0; k < npX; k += 32) {
                    const bool v2 = k + 16 < npX;
                    int j1, j2;
                    float w1, w2;
                    pair_of(k, j1, w1);
                    if (v2) pair_of(k + 16, j2, w2);
                    else { j2 = j1; w2 = 0.f; }
                    const uint4 sj1 = a.s4[j1];
                    const int2 tj1 = a.tm[j1];
                    const uint4 sj2 = a.s4[j2];
                    const int2 tj2 = a.tm[j2];
                    mixed_term(sX, kqX, tiX, sj1, tj1, w1, ff);
                    if (v2) mixed_term(sX, kqX, tiX, sj2, tj2, w2, ff);
                }
                // sums over each half-warp
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int o = 8; o >= 1; o >>= 1) ff[q] += __shfl_xor_sync(FULL, ff[q], o);
                if (l16 == 0 && (!hb || hasB)) {
                    float* Fr = reinterpret_cast<float*>(a.F_real) + 3 * (size_t)(hb ? iB : iA);
                    Fr[0] = ff[0];
                    Fr[1] = ff[1];
                    Fr[2] = ff[2];
                    facc_f[0] += ff[0]; facc_f[1] += ff[1]; facc_f[2] += ff[2];
                }
                flush_sums(hasB ? 2 : 1);

                // ---- debug record (caller index order) ---------------------------
                if (a.debug) {
                    for (int x = 0; x < (hasB ? 2 : 1); ++x) {
                        const int ix = x ? iB : iA, gx = a.perm[ix];
                        const int ncx = x ? ncB : ncA, ncxc = x ? ncBc : ncAc, nsx = x ? nsB : nsA;
                        const int nbx = x ? nbB : nbA;
                        const int* cx_ = x ? coreB : coreA;
                        const int* jx = x ? jB : jA;
                        if (lane == 0) { a.dbg_ncore[gx] = ncx; a.dbg_nshell[gx] = nsx; }
                        for (int t = lane; t < a.dbg_cap; t += 32)
                            a.dbg_core[(size_t)gx * a.dbg_cap + t] = t < ncxc ? a.perm[cx_[t]] : -1;
                        for (int k = lane; k < p; k += 32)
                            a.dbg_batch[(size_t)gx * p + k] = k < nbx ? a.perm[jx[k]] : -1;
                    }
                }
                __syncwarp();
            }
        } else {
            int kloc = 0;
            for (int i = A0 + wib; i < A1; i += WARPS, ++kloc) {
                // Philox words of the shell slots, made for lay.ga atoms per pass:
                // slot k of atom gi uses word k%4 of the block at (gi, k/4, step, 1)
                const int aslot = kloc % lay.ga;
                if (aslot == 0) {
                    __syncwarp();
                    for (int t = lane; t < lay.ga * nbk; t += 32) {
                        const int aa = t / nbk, b = t - aa * nbk;
                        const int ii = i + WARPS * aa;
                        if (ii < A1) {
                            uint64_t w[4];
                            philox4x64_10((uint64_t)a.perm[ii], (uint64_t)b, a.step, 1ull, c.seed, 0ull, w);
#pragma unroll
                            for (int qd = 0; qd < 4; ++qd) words[aa * p_pad + 4 * b + qd] = w[qd];
                        }
                    }
                    __syncwarp();
                }
                one_atom(i, words + (size_t)aslot * p_pad);
            }
        }
    }

    // every staging copy has completed (each unit waited for its phase): the
    // barrier is invalidated before its memory is initialised again (the
    // batched form runs this body once per task)
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&s_mbar);

    // ---- deterministic block partials ---------------------------------------
    if constexpr (LMODE == RBL_BUILD) return;        // no pair terms in the list build
    if (MIXED) {
#pragma unroll
        for (int q = 0; q < 3; ++q) acc_e[q] += (double)facc_e[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) acc_w[q] += (double)facc_w[q];
#pragma unroll
        for (int q = 0; q < 3; ++q) acc_f[q] += (double)facc_f[q];
    }
    double v[RBE_NPART_RBL] = {acc_e[0], acc_e[1], acc_e[2], acc_w[0], acc_w[1], acc_w[2],
                               acc_w[3], acc_w[4], acc_w[5], acc_f[0], acc_f[1], acc_f[2]};
#pragma unroll
    for (int q = 0; q < RBE_NPART_RBL; ++q) v[q] = warp_sum(v[q]);
    __syncthreads();
    if (lane == 0)
        for (int q = 0; q < RBE_NPART_RBL; ++q) red[wib][q] = v[q];
    __syncthreads();
    if (threadIdx.x < RBE_NPART_RBL) {
        double s = 0.0;
        for (int w = 0; w < WARPS; ++w) s += red[w][threadIdx.x];
        a.part[(size_t)slot * RBE_NPART_RBL + threadIdx.x] = s;
    }
    if (ADJ)
        for (int t = threadIdx.x; t < 4 * nt2; t += blockDim.x)
            a.part_lj[(size_t)slot * 4 * nt2 + t] = s_glj[t];
}

template <bool MIXED, bool SMALL, bool ADJ>
__global__ void __launch_bounds__(WARPS * 32, RBE_BLOCKS_RBL) k_rbl(RblArgs a)
{
    rbl_body<MIXED, SMALL, ADJ>(a, blockIdx.x, gridDim.x);
}

// Verlet-skin variant: the stored lists from the stencil walk at r_s + skin
// (a.c and a.g hold that radius and its geometry), and the per-step kernel
// over the stored lists.
template <bool SMALL>
__global__ void __launch_bounds__(WARPS * 32, RBE_BLOCKS_RBL) k_rbl_build(RblArgs a)
{
    rbl_body<false, SMALL, false, RBL_BUILD>(a, blockIdx.x, gridDim.x);
}

template <bool MIXED>
__global__ void __launch_bounds__(WARPS * 32, RBE_BLOCKS_STORED) k_rbl_stored(RblArgs a)
{
    rbl_body<MIXED, false, false, RBL_STORED>(a, blockIdx.x, gridDim.x);
}

// Pair kernel over many systems.  PERSIST: a grid of resident blocks, each
// repeatedly taking the next (replica, slot) task from a queue ordered by
// decreasing estimated cost; otherwise one block per task in that order (the
// hardware block scheduler then hands them out in the same order).  A block
// copies its replica's arguments to shared memory and runs the slot.  A
// slot's result does not depend on which block runs it, so the partials, and
// every force and energy, equal those of the single-system launch.
static_assert(sizeof(RblArgs) % 8 == 0, "RblArgs copy");
template <bool MIXED, bool PERSIST>
__global__ void __launch_bounds__(WARPS * 32, RBE_BLOCKS_RBL) k_rbl_batch(const RblArgs* __restrict__ args,
                                                             const int2* __restrict__ tasks, int ntasks,
                                                             BatchCtl* __restrict__ ctl)
{
    __shared__ __align__(16) RblArgs s_a;
    __shared__ int s_task;
    for (int iter = 0;; ++iter) {
        if (!PERSIST && iter > 0) break;
        __syncthreads();                       // the previous task is done with s_a
        if (threadIdx.x == 0) s_task = PERSIST ? atomicAdd(&ctl->rbl_next, 1) : (int)blockIdx.x;
        __syncthreads();
        const int t = s_task;
        if (t >= ntasks) break;
        const int2 tk = tasks[t];
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(args + tk.x);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_a);
        for (int k = threadIdx.x; k < (int)(sizeof(RblArgs) / 8); k += blockDim.x) dst[k] = src[k];
        __syncthreads();
        if (threadIdx.x == 0) s_a.step = ctl->step;
        __syncthreads();
        if (s_a.g.small) rbl_body<MIXED, true, false>(s_a, tk.y, s_a.nslots);
        else rbl_body<MIXED, false, false>(s_a, tk.y, s_a.nslots);
    }
}

template <bool MIXED, bool SMALL, bool ADJ>
void launch_t(rbe_ctx* ctx, const RblArgs& a, int smem, cudaStream_t st)
{
    cudaFuncSetAttribute(k_rbl<MIXED, SMALL, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_rbl<MIXED, SMALL, ADJ><<<ctx->grid_rbl, WARPS * 32, smem, st>>>(a);
}

template <bool MIXED, bool SMALL>
int occupancy_t(int smem)
{
    int nb = 0, nb2 = 0;
    cudaFuncSetAttribute(k_rbl<MIXED, SMALL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rbl<MIXED, SMALL, false>, WARPS * 32, smem);
    cudaFuncSetAttribute(k_rbl<MIXED, SMALL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_rbl<MIXED, SMALL, true>, WARPS * 32, smem);
    return nb < nb2 ? nb : nb2;
}

}  // namespace

int rbl_smem_bytes(const rbe_ctx* ctx)
{
    int nt2 = ctx->c.ntypes * ctx->c.ntypes;
    return (int)smem_layout(ctx->rbl, nt2, ctx->c.p, ctx->core_cap, ctx->shell_cap).total;
}

size_t rbl_args_bytes() { return sizeof(RblArgs); }

// Dynamic shared memory per block that leaves room for RBE_BLOCKS_RBL resident
// blocks of every form of the pair kernel on the current device: that share
// of the SM's shared memory, less the per-block reservation and the largest
// static shared memory of the forms (the batched form also keeps its
// arguments there).
int rbl_smem_target()
{
    static int cached = 0;
    if (cached > 0) return cached;
    int dev = 0, per_sm = 0, reserved = 0;
    cudaFuncAttributes f1, f2;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&f1, k_rbl<true, false, false>) != cudaSuccess ||
        cudaFuncGetAttributes(&f2, k_rbl_batch<true, true>) != cudaSuccess) {
        cudaGetLastError();
        return 110 * 1024;
    }
    const size_t st = f1.sharedSizeBytes > f2.sharedSizeBytes ? f1.sharedSizeBytes : f2.sharedSizeBytes;
    cached = per_sm / RBE_BLOCKS_RBL - reserved - (int)st;
    return cached;
}

void rbl_fill_args(const rbe_ctx* ctx, int n, void* out)
{
    RblArgs& a = *static_cast<RblArgs*>(out);
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.step = 0;
    a.s4 = ctx->s4; a.f4 = ctx->f4; a.p4 = ctx->p4; a.tm = ctx->tm; a.perm = ctx->perm;
    a.cell_start = ctx->cell_start;
    a.lj = ctx->lj; a.F_real = ctx->F_real; a.part = ctx->part_rbl; a.status = ctx->status;
    a.c = ctx->c;
    a.g = ctx->rbl;
    a.core_cap = ctx->core_cap; a.shell_cap = ctx->shell_cap;
    a.debug = ctx->debug; a.dbg_cap = ctx->dbg_cap_core;
    a.dbg_ncore = ctx->dbg_ncore; a.dbg_nshell = ctx->dbg_nshell; a.dbg_core = ctx->dbg_core; a.dbg_batch = ctx->dbg_batch;
    a.dbg_unstaged = ctx->dbg_unstaged;
    a.vs = ctx->vs; a.vbar = ctx->totals + 16; a.gq_own = ctx->gq_own; a.gq_tr = ctx->gq_tr; a.part_lj = ctx->part_lj;
    a.nslots = ctx->grid_rbl;
}

long rbl_units(const rbe_ctx* ctx)
{
    const int nc = ctx->c.n_cell, G = ctx->rbl.G;
    return (long)nc * nc * ((nc + G - 1) / G);
}

void launch_rbl(rbe_ctx* ctx, int n, uint64_t step, cudaStream_t st, bool adjoint)
{
    RblArgs a;
    rbl_fill_args(ctx, n, &a);
    a.step = step;
    if (adjoint) a.debug = 0;
    if (a.debug) cudaMemsetAsync(ctx->dbg_unstaged, 0, 2 * sizeof(int), st);
    int smem = rbl_smem_bytes(ctx);
    prof_begin(ctx, RBE_K_RBL, st);
    const bool small = ctx->rbl.small;
    const bool mixed = ctx->precision == RBE_MIXED;
    if (adjoint) {
        if (mixed) { if (small) launch_t<true, true, true>(ctx, a, smem, st); else launch_t<true, false, true>(ctx, a, smem, st); }
        else { if (small) launch_t<false, true, true>(ctx, a, smem, st); else launch_t<false, false, true>(ctx, a, smem, st); }
    } else {
        if (mixed) { if (small) launch_t<true, true, false>(ctx, a, smem, st); else launch_t<true, false, false>(ctx, a, smem, st); }
        else { if (small) launch_t<false, true, false>(ctx, a, smem, st); else launch_t<false, false, false>(ctx, a, smem, st); }
    }
    prof_end(ctx, RBE_K_RBL, st);
}

// (the list build keeps no core list in shared memory: members go straight
// to the stored lists)
int rbl_build_smem_bytes(const rbe_ctx* ctx)
{
    return (int)smem_layout(ctx->skin_g, ctx->c.ntypes * ctx->c.ntypes, ctx->c.p, 0, 32).total;
}

long rbl_build_units(const rbe_ctx* ctx)
{
    const int nc = ctx->c.n_cell, G = ctx->skin_g.G;
    return (long)nc * nc * ((nc + G - 1) / G);
}

// Stored lists V(i) of the Verlet-skin variant from the sorted arrays of the
// rebuild step: the stencil walk with both radii set to r_s + skin.
void launch_rbl_build(rbe_ctx* ctx, int n, cudaStream_t st)
{
    RblArgs a;
    rbl_fill_args(ctx, n, &a);
    a.c = ctx->skin_c;
    a.g = ctx->skin_g;
    a.core_cap = ctx->skin_vcap;
    a.shell_cap = 32;
    a.vlist = ctx->vlist; a.vcnt = ctx->vcnt; a.vcap = ctx->skin_vcap;
    a.debug = 0;
    a.nslots = ctx->skin_grid_build;
    const int smem = rbl_build_smem_bytes(ctx);
    prof_begin(ctx, RBE_K_SKIN, st);
    if (ctx->skin_g.small) {
        cudaFuncSetAttribute(k_rbl_build<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_rbl_build<true><<<ctx->skin_grid_build, WARPS * 32, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(k_rbl_build<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_rbl_build<false><<<ctx->skin_grid_build, WARPS * 32, smem, st>>>(a);
    }
    prof_end(ctx, RBE_K_SKIN, st);
}

// Lists, batches and pair terms of one step from the stored lists (same
// grid and block partials as the stencil launch, so finalisation is shared).
void launch_rbl_stored(rbe_ctx* ctx, int n, uint64_t step, cudaStream_t st)
{
    RblArgs a;
    rbl_fill_args(ctx, n, &a);
    a.step = step;
    RblGeom g = ctx->rbl;
    g.G = 1; g.nrows = 0; g.cap_stage = 0; g.cells_per_row = 0; g.small = 0;
    a.g = g;
    a.vlist = ctx->vlist; a.vcnt = ctx->vcnt; a.vcap = ctx->skin_vcap;
    const int smem =
        (int)smem_layout(g, ctx->c.ntypes * ctx->c.ntypes, ctx->c.p, ctx->core_cap, ctx->shell_cap, true).total;
    if (a.debug) cudaMemsetAsync(ctx->dbg_unstaged, 0, 2 * sizeof(int), st);
    prof_begin(ctx, RBE_K_RBL, st);
    if (ctx->precision == RBE_MIXED) {
        cudaFuncSetAttribute(k_rbl_stored<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_rbl_stored<true><<<ctx->grid_rbl, WARPS * 32, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(k_rbl_stored<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_rbl_stored<false><<<ctx->grid_rbl, WARPS * 32, smem, st>>>(a);
    }
    prof_end(ctx, RBE_K_RBL, st);
}

int rbl_blocks_per_sm(const rbe_ctx* ctx)
{
    int smem = rbl_smem_bytes(ctx);
    const bool small = ctx->rbl.small;
    int nb;
    if (ctx->precision == RBE_MIXED) nb = small ? occupancy_t<true, true>(smem) : occupancy_t<true, false>(smem);
    else nb = small ? occupancy_t<false, true>(smem) : occupancy_t<false, false>(smem);
    return nb > 0 ? nb : 1;
}

namespace {
template <bool MIXED, bool PERSIST>
int occ_batch(int smem)
{
    int nb = 0;
    cudaFuncSetAttribute(k_rbl_batch<MIXED, PERSIST>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rbl_batch<MIXED, PERSIST>, WARPS * 32, smem);
    return nb;
}
}  // namespace

int rbl_max_blocks_per_sm(int precision, int smem)
{
    int a, b;
    if (precision == RBE_MIXED) { a = occ_batch<true, true>(smem); b = occ_batch<true, false>(smem); }
    else { a = occ_batch<false, true>(smem); b = occ_batch<false, false>(smem); }
    return a < b ? a : b;
}

void launch_rbl_batch(const BatchPlan& bp, cudaStream_t st)
{
    const RblArgs* args = static_cast<const RblArgs*>(bp.rbl_args);
    const int grid = bp.rbl_persistent ? bp.rbl_grid : bp.ntasks;
    if (bp.precision == RBE_MIXED) {
        if (bp.rbl_persistent)
            k_rbl_batch<true, true><<<grid, WARPS * 32, bp.rbl_smem, st>>>(args, bp.tasks, bp.ntasks, bp.ctl);
        else
            k_rbl_batch<true, false><<<grid, WARPS * 32, bp.rbl_smem, st>>>(args, bp.tasks, bp.ntasks, bp.ctl);
    } else {
        if (bp.rbl_persistent)
            k_rbl_batch<false, true><<<grid, WARPS * 32, bp.rbl_smem, st>>>(args, bp.tasks, bp.ntasks, bp.ctl);
        else
            k_rbl_batch<false, false><<<grid, WARPS * 32, bp.rbl_smem, st>>>(args, bp.tasks, bp.ntasks, bp.ctl);
    }
}
