/*
 * rbe.h -- C ABI of librbe.so: the improved random batch Ewald (IRBE) non-bonded
 * force step of Liang, Xu & Zhao (arXiv 2204.13595) on one NVIDIA GB300
 * (sm_103a).
 *
 * The step joins two stochastic estimators:
 *   RBL (Sec. 2.3, Eqs. (2.10)-(2.13)): every pair inside the core radius r_c
 *       is summed exactly; a batch of p atoms drawn from the shell
 *       r_c < r <= r_s is summed with weight N_S/p; the mean net real-space
 *       force is removed from every atom (momentum correction, Eq. (2.13)).
 *   RBE (Sec. 2.2, Eqs. (2.6)-(2.9)): P wave vectors k != 0 are drawn from
 *       P_k = exp(-k^2/(4 alpha))/S, the structure factors
 *       rho(k) = sum_j q_j exp(i k.r_j) are formed over all atoms and each
 *       atom's long-range force is summed over the batch.
 *
 * Notation: r_c here is the paper's core radius r_eta and r_s the paper's
 * outer cutoff r_c; p is the paper's shell batch p~ and P its Fourier batch p.
 *
 * Every random draw is a pure function of (seed, step, atom, slot) through
 * Philox4x64-10: key (seed, 0); shell slot k of atom i uses word k%4 of the
 * block at counter (i, k/4, step, 1), where i is the caller's atom index;
 * k sample l, attempt t uses words 0..2 of the block at counter (l, t, step, 2).
 * List membership is decided on 32-bit fixed-point fractional coordinates
 * s = floor(frac(x/L) 2^32) with exact integer squared distances, so lists and
 * batches are reproducible bit for bit.  Shell ordinals index S(i) in the
 * canonical order: ascending (cell, fixed-point x code s_x, atom index) on the
 * grid of floor(L/r_c) cells per axis (the cell grid of Sec. 2.3).
 *
 * Conventions for every entry point:
 *   - return 0 (RBE_OK) or a negative RBE_E* code; no exception or abort
 *     crosses the ABI; rbe_last_error() gives a message for the last failure;
 *   - a context is not thread-safe: use one context per host thread/stream;
 *   - array arguments are caller-owned; the library never frees them;
 *   - pos is [n][3] row-major FP64 (Angstrom or sigma), q is [n] FP64,
 *     type and mol are [n] int32; F and vel are [n][3] FP64;
 *   - a cuda_stream argument is a cudaStream_t (NULL = legacy default stream);
 *     work is enqueued on it and the call returns without waiting, unless a
 *     host pointer is involved (see rbe_forces).
 */
#ifndef RBE_H
#define RBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RBE_OK            0
#define RBE_EINVAL       -1   /* bad parameter or argument                     */
#define RBE_ENONNEUTRAL  -2   /* |sum q| > 1e-10 sum |q| (Sec. 2.1 assumes 0)  */
#define RBE_EOVERLAP     -3   /* two atoms at the same fixed-point position     */
#define RBE_ENONFINITE   -4   /* non-finite position or result                  */
#define RBE_ECAPACITY    -5   /* a per-atom list exceeded its capacity          */
#define RBE_ECUDA        -6   /* a CUDA runtime call failed, or a device-side
                                  copy wait ran out (shared-memory staging)    */
#define RBE_ENOMEM       -7   /* device allocation failed                       */

/* precision modes (rbe_set_precision) */
#define RBE_FP64   0   /* all arithmetic in FP64                                */
#define RBE_MIXED  1   /* FP32 pair and phase arithmetic; FP64 positions,
                          rho(k) accumulation, force and energy totals          */

/* energy components written by rbe_forces (RBE_NE doubles) */
#define RBE_NE 6
#define RBE_E_REAL   0   /* erfc real-space Coulomb, RBL estimate (Eq. (2.3) U^short) */
#define RBE_E_KSPACE 1   /* reciprocal space, RBE estimate (Eq. (2.3) U^long)         */
#define RBE_E_SELF   2   /* -k_e sqrt(alpha/pi) sum q^2 (Eq. (2.3) U^corr)             */
#define RBE_E_LJ     3   /* Lennard-Jones, RBL estimate (Eq. (2.3) U^lj)               */
#define RBE_E_EXCL   4   /* -k_e q_i q_j erf(sqrt(alpha) r)/r over same-molecule pairs */
#define RBE_E_BOND   5   /* harmonic water bonds and angles (rbe_set_water_bonds)      */
/* virial components (RBE_NW doubles): xx yy zz xy xz yz of
 * W = -1/2 sum_i sum_j w_ij r_ij (x) f_ij  (r_ij = r_j - r_i, w_ij the RBL
 * weight) plus the reweighted reciprocal-space Ewald virial; non-bonded only. */
#define RBE_NW 6

typedef struct rbe_ctx rbe_ctx;

/* Creates a context for a cubic periodic box of edge box_L (Sec. 2.1).
 * alpha > 0 is the Ewald parameter of erfc(sqrt(alpha) r) and
 * exp(-k^2/(4 alpha)) (Eqs. (2.2)-(2.3)); 0 < r_c < r_s <= box_L/2 are the
 * core radius and outer cutoff (Sec. 2.3); p >= 1 the shell batch size
 * (Eq. (2.11)); P >= 1 the Fourier batch size (Eq. (2.9)); seed the Philox
 * key.  Coulomb prefactor defaults to 1, no LJ, precision RBE_FP64.
 * Allocates device memory lazily on the first rbe_forces call, on the device
 * current at that time.  *out receives the context (NULL on failure). */
int rbe_create(rbe_ctx** out, double box_L, double alpha, double r_c, double r_s,
               int p, int P, uint64_t seed);

/* Coulomb prefactor k_e multiplying every q_i q_j term (the paper writes
 * Gaussian units, Eq. (2.1)): 1.4 for the reduced electrolyte, 1389.35458
 * kJ mol^-1 A e^-2 for water. */
int rbe_set_coulomb(rbe_ctx* ctx, double k_e);

/* Lennard-Jones per-type parameters (host arrays of ntypes <= 16 entries)
 * mixed by Lorentz-Berthelot (sigma_ij = (sigma_i+sigma_j)/2,
 * eps_ij = sqrt(eps_i eps_j)); the pair force is Eq. (2.10), truncated at
 * r_s; shift_energy = 1 shifts the LJ energy to zero at r_s. */
int rbe_set_lj(rbe_ctx* ctx, int ntypes, const double* eps, const double* sigma, int shift_energy);

/* RBE_FP64 or RBE_MIXED. */
int rbe_set_precision(rbe_ctx* ctx, int mode);

/* Harmonic 3-site water bonded terms for molecules m = 0..n_mol-1 made of
 * atoms (3m, 3m+1, 3m+2) = (O, H, H): U = 1/2 k_b (r - r0)^2 per O-H bond and
 * 1/2 k_theta (theta - theta0)^2 per H-O-H angle (theta in radians).  Added by
 * rbe_forces to F and to energy[RBE_E_BOND].  n_mol = 0 disables them.
 * The paper integrates with a force field (Sec. 3.2); these constants are the
 * caller's choice. */
int rbe_set_water_bonds(rbe_ctx* ctx, int n_mol, double k_b, double r0, double k_theta, double theta0);

/* Per-atom list capacities used by the pair kernel (0 = automatic, from the
 * density: roughly twice the mean count plus a margin).  A list longer than its
 * capacity sets RBE_ECAPACITY in the status word and records the count met;
 * the overflowing evaluation's forces are then wrong.  rbe_forces calls that
 * wait (host pointers or host energy/virial) retry once with capacities that
 * hold the counts met, rbe_step retries the failing step once the same way,
 * and rbe_sync_status, when it reports RBE_ECAPACITY, grows the capacities
 * for the next call.  Capacities that shared memory cannot hold give
 * RBE_ECAPACITY from the next call. */
int rbe_set_capacity(rbe_ctx* ctx, int core_cap, int shell_cap);

/* One IRBE force evaluation at MD step `step` (Algorithm 1, force steps):
 * F = F^core + F^{shell,*} - F^corr + F^{long,*} (Eqs. (2.9), (2.11), (2.13))
 * plus the water bonded terms when configured.  Excluded pairs are the pairs
 * with equal mol id (mol may be NULL: no exclusions); they keep their set
 * membership and contribute -k_e q_i q_j erf(sqrt(alpha) r)/r instead of
 * erfc + LJ.  type may be NULL (all type 0).
 * pos, q, type, mol, F are either all device pointers or all host pointers.
 * With host pointers the call returns after F is written: inputs in pinned
 * (page-locked, device-mapped) host memory are read by the device in place,
 * other host inputs are first copied to device memory (as are all host inputs
 * of a context with a Verlet skin); F is computed in device memory and copied
 * back.  energy (RBE_NE) and virial (RBE_NW) may each
 * be NULL, a host pointer (the call then waits for the stream) or a device
 * pointer.  Positions need not be wrapped into the box.
 * Errors found on the device (overlap, capacity, non-neutral charge,
 * non-finite input) are latched in a status word read by rbe_sync_status();
 * a call that waits reads it itself and retries a capacity overflow once
 * (rbe_set_capacity), leaving other errors latched. */
int rbe_forces(rbe_ctx* ctx, uint64_t step, int n, const double* pos, const double* q,
               const int32_t* type, const int32_t* mol, double* F, double* energy, double* virial,
               void* cuda_stream);

/* nsteps of velocity Verlet (Algorithm 1, integration step, NVE):
 *   v += (dt/2) accel F/m;  x += dt v;  F = rbe_forces(step0+k+1);  v += (dt/2) accel F/m
 * accel converts force/mass to acceleration (1 in reduced units, 1e-4 for
 * kJ/mol/A, g/mol, fs).  On entry F must hold the forces at (pos, step0); on
 * exit it holds those at the final positions.  All arrays are device pointers;
 * energy_trace (device, may be NULL) receives per step the potential energy
 * (sum of the RBE_NE components) and the kinetic energy / accel.
 * The call waits for the stream at its end.  An error latched on the device
 * stops the integration there: the kicks of that and every later step leave
 * positions and velocities as they are (a status latched before the call and
 * not read stops it at its first step).  A capacity overflow in the force
 * evaluation of a step is retried once: the capacities are grown to the
 * counts met, that evaluation and the step's second half kick are redone and
 * the remaining steps run.  Any other error, or a second overflow, is
 * returned (and stays latched for rbe_sync_status); positions, velocities
 * and F are then the state at the force evaluation that failed, whose step
 * rbe_get_info reports (out[9]); the energy_trace entries from that step on
 * are not meaningful. */
int rbe_step(rbe_ctx* ctx, uint64_t step0, int nsteps, double dt, double accel, int n,
             double* pos, double* vel, const double* mass, const double* q, const int32_t* type,
             const int32_t* mol, double* F, double* energy_trace, void* cuda_stream);

/* Gradients of the force step at MD step `step` with its random draws frozen
 * (the same lists, shell batches and k samples as rbe_forces at that step;
 * the paper's estimator, Eqs. (2.9)-(2.13), differentiated term by term):
 *   dEdq[n]   = dE/dq_i, E the sum of the RBE_E_REAL..RBE_E_EXCL components;
 *   dLdq[n]   = dL/dq_i with L = sum_i gF_i . F_i (a vector-Jacobian product
 *               of the non-bonded force; gF may be NULL for L = 0);
 *   dEdeps, dEdsig, dLdeps, dLdsig [ntypes] = the same w.r.t. the per-type
 *               LJ parameters through Lorentz-Berthelot mixing (host arrays;
 *               the call waits; a type with eps = 0 paired with eps > 0 has
 *               an infinite eps derivative, reported as HUGE_VAL).
 * pos, q, type, mol, gF, dEdq, dLdq are device pointers; any output may be
 * NULL.  Pair terms are recomputed, not stored; the part of a pair that
 * belongs to the other atom's charge is added atomically, so dEdq and dLdq
 * are exact to rounding but not bitwise reproducible run to run. */
int rbe_adjoint(rbe_ctx* ctx, uint64_t step, int n, const double* pos, const double* q, const int32_t* type,
                const int32_t* mol, const double* gF, double* dEdq, double* dLdq, double* dEdeps, double* dEdsig,
                double* dLdeps, double* dLdsig, void* cuda_stream);

/* Waits for cuda_stream, returns the first latched device error (or RBE_OK)
 * and clears the status word; after RBE_ECAPACITY the next call uses
 * capacities that hold the counts met.  An evaluation whose input holds a non-finite
 * position latches RBE_ENONFINITE and its result is undefined; such atoms are
 * placed on a lattice at the system's density for the rest of that step, so a
 * run that has blown up costs what a normal step costs until it is stopped. */
int rbe_sync_status(rbe_ctx* ctx, void* cuda_stream);

/* Debug recording: when on, rbe_forces also records per atom (indexed by the
 * caller's atom index) |C(i)|, |S(i)|, the core ids in canonical order (up to
 * cap_core) and the batch B(i) in slot order (p entries, -1 padded). */
int rbe_set_debug(rbe_ctx* ctx, int on, int cap_core);

/* Copies the lists recorded by the last rbe_forces with debug on into host
 * arrays: n_core[n], n_shell[n], core[n][cap_core], batch[n][p] (any may be
 * NULL).  Waits for cuda_stream. */
int rbe_get_lists(rbe_ctx* ctx, int n, int32_t* n_core, int32_t* n_shell, int32_t* core,
                  int32_t* batch, void* cuda_stream);

/* Copies the last step's k samples m[P][3] (integers, k = 2 pi m / L) and
 * structure factors rho[P][2] (re, im) into host arrays (either may be NULL).
 * Waits for cuda_stream. */
int rbe_get_kspace(rbe_ctx* ctx, int32_t* m, double* rho, void* cuda_stream);

/* Derived parameters: out[0] cells per axis, out[1] stencil reach in cells,
 * out[2] k truncation M, out[3] S = H^3 - 1 (Eq. (2.6)), out[4] core capacity,
 * out[5] shell capacity (after the last rbe_forces), out[6] kernel launches
 * of the last rbe_forces, out[7] work units of the last pair-kernel launch
 * whose stencil exceeded the shared-memory staging capacity and was read
 * from global memory, out[8] (atom, pass of 32 stencil rows) pairs of that
 * launch whose candidates (more than 2048) were classified range by range
 * instead of as one concatenated list (both counted with rbe_set_debug on;
 * -1 otherwise), out[9] the step whose force evaluation stopped the last
 * rbe_step (-1 if it ran to the end), out[10] the stored-list rebuilds of the
 * Verlet skin so far, out[11] the entries per stored list. */
int rbe_get_info(rbe_ctx* ctx, double* out, int nout);

/* Kernel timing: when on, every launch is bracketed by CUDA events on its
 * stream, and a force evaluation runs all its kernels on the caller's stream
 * (otherwise the k sampling and structure factors run on an auxiliary stream
 * beside the pair kernel, where their event intervals would include waits
 * for SMs).  rbe_get_profile waits for cuda_stream and returns, per kernel id
 * (RBE_K_*), the summed milliseconds and the number of launches since the
 * last reset (reset = 1 clears them afterwards). */
#define RBE_K_QUANTIZE 0
#define RBE_K_SCAN     1
#define RBE_K_SCATTER  2
#define RBE_K_SORT     3
#define RBE_K_GATHER   4
#define RBE_K_KSAMPLE  5
#define RBE_K_RHO      6
#define RBE_K_RHOSUM   7
#define RBE_K_RBL      8
#define RBE_K_BONDED   9
#define RBE_K_FINAL    10
#define RBE_K_KFORCE   11
#define RBE_K_VV       12
#define RBE_K_MISC     13
#define RBE_K_SKIN     14   /* stored-list build and rebuild test of the Verlet skin */
#define RBE_NKERNELS   15
int rbe_set_profiling(rbe_ctx* ctx, int on);
int rbe_get_profile(rbe_ctx* ctx, double* ms, int64_t* launches, int reset, void* cuda_stream);

const char* rbe_last_error(const rbe_ctx* ctx);

/* Structure factors rho_l = sum_j q_j exp(i k_l . r_j), k_l = 2 pi m_l / box_L,
 * for P given integer vectors m[P][3], from n atoms pos[n][3], q[n]; writes
 * rho[P][2] (re, im).  FP64: the phase (m . x)/L is reduced to [-1/2, 1/2]
 * and evaluated with sincospi.  This is the structure factor of the context
 * path (rbe_get_kspace) by other arithmetic (the context path takes the
 * phase from 32-bit fixed-point codes): the two agree to about 1e-13 of
 * sum |q|, not bit for bit.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let the library allocate device memory (their device memory is
 * owned by another allocator or a fixed budget, or allocation and its
 * implicit synchronisation are not allowed where they call).  It allocates
 * nothing: its scratch is a static device array of RBE_NOALLOC_BLOCKS x
 * RBE_NOALLOC_PMAX complex partial sums (2 MiB) that every GPU loading the
 * library holds until the process exits.  All pointers are device pointers
 * owned by the caller; work is enqueued on cuda_stream and the call returns
 * without waiting.  The first call on a device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture.  Calls share the array: calls whose kernels overlap on the GPU
 * race.  Returns RBE_EINVAL for bad arguments, RBE_ELIMIT when P exceeds
 * RBE_NOALLOC_PMAX, RBE_ECUDA when the set-up or a launch fails (a launch
 * error the caller left pending is also reported, and cleared, here).  The
 * device address is looked up once per device and not refreshed after
 * cudaDeviceReset: do not call this entry point on a device after resetting
 * it. */
#define RBE_ELIMIT        -8   /* size beyond a compiled maximum                */
#define RBE_NOALLOC_BLOCKS 256
#define RBE_NOALLOC_PMAX   512
int rbe_rho_noalloc(int n, const double* pos, const double* q, double box_L, int P, const int32_t* m,
                    double* rho, void* cuda_stream);

/* Releases the context and its device memory (after the caller's streams are
 * idle). */
void rbe_destroy(rbe_ctx* ctx);

/* Variants of the method (the paper leaves them open; defaults = base method).
 *
 * Shell batch (Algorithm 1, shell selection step): RBE_SHELL_FLOYD draws the
 * min(p, N_S) atoms of B(i) without replacement (Floyd's algorithm over the
 * shell ordinals); RBE_SHELL_REPLACE draws, when N_S > p, p independent
 * uniform ordinals (slot k: floor(u_k N_S / 2^64), u_k the slot's Philox
 * word), weight N_S/p, repeats allowed. */
#define RBE_SHELL_FLOYD   0
#define RBE_SHELL_REPLACE 1
int rbe_set_shell_sampling(rbe_ctx* ctx, int mode);

/* LJ cutoff per pair type: factor f > 0 truncates the LJ term of pair (a, b)
 * at min(f sigma_ab, r_s), shifted to zero there when rbe_set_lj's
 * shift_energy is set; f = 2^(1/6) with the shift is the WCA soft sphere of
 * the paper's primitive-model electrolytes (Sec. 3.1, "shifted-truncated
 * LJ").  f = 0 (default): LJ to r_s.  Pairs beyond the cutoff keep their
 * Coulomb term. */
int rbe_set_lj_cutoff(rbe_ctx* ctx, double factor);

/* k-sample pool (Algorithm 1, pool step; Sec. 2.2): size K > 0 builds, once,
 * a pool of K wave vectors from one Metropolis-Hastings chain per axis
 * (target the discrete Gaussian of Eq. (2.8); proposal round(x),
 * x ~ N(0, alpha L^2 / (2 pi^2)); chain iteration t of axis a uses Philox
 * block (t, a, 0, 4); burn_in iterations discarded; k = 0 skipped), and each
 * step's sample l is pool entry floor(u K / 2^64), u word 0 of block
 * (l, 0, step, 5).  K = 0 (default): fresh exact draws every step. */
int rbe_set_kpool(rbe_ctx* ctx, int size, int burn_in);

/* Langevin thermostat for rbe_step and rbe_batch_step (Sec. 3.1 runs its
 * electrolytes with a Langevin thermostat of relaxation time tau inside
 * velocity Verlet).  With tau > 0, every force evaluation at step s adds
 *   F^L_i = -(m_i / (accel tau)) v_i + sqrt(24 m_i kT / (accel tau dt)) (u - 1/2)
 * per component, v_i the velocity after the first half kick and u uniform in
 * [0, 1) from word a of the Philox block at counter (i, 0, s, 3) (i the
 * caller's atom index): friction plus a uniform random force of variance
 * 2 m kT / (accel tau dt); the next step's first half kick uses the same F^L.
 * kT is in the caller's energy units.  tau <= 0 (default) turns it off (NVE).
 * F returned by rbe_step stays the conservative force. */
int rbe_set_langevin(rbe_ctx* ctx, double kT, double tau);

/* Resume support for thermostatted runs.  The state of a velocity-Verlet run
 * at step s is (pos, vel, F, s) and, with the thermostat, the Langevin force
 * F^L made at step s, which the first half kick of step s + 1 uses.  An
 * rbe_step (or rbe_batch_step) call that starts at the step where the
 * context's previous run ended reuses the held F^L, so a run split into
 * several calls equals one call bit for bit; a call that starts anywhere else
 * makes F^L from the entry velocities.  For a checkpoint, get copies the held
 * F^L ([n][3], any host or device pointer) and its step (RBE_EINVAL if none is
 * held for n atoms); set installs them in a context (e.g. a fresh one after a
 * restart), so that resuming at that step is exact. */
int rbe_get_langevin_force(rbe_ctx* ctx, int n, double* FL, uint64_t* step);
int rbe_set_langevin_force(rbe_ctx* ctx, int n, const double* FL, uint64_t step);

/* Verlet skin (Sec. 2.3 remarks that a cell edge slightly above r_eta spares
 * rebuilding the lists every step; the scheme is this library's): with
 * skin > 0 the context keeps, per atom, a stored list V(i) of every atom
 * within r_s + skin at the positions of the last rebuild, in the canonical
 * order of that step (ascending cell, fixed-point x, atom index).  Each force
 * evaluation classifies V(i) by the exact rule at the current positions, so
 * C(i) and S(i) are those of the stencil walk; the shell ordinals of the
 * batch follow the order of V(i).  The atoms keep the sorted order of the
 * rebuild between rebuilds.  A rebuild happens on the first call, when n or
 * the skin changes, and when some atom has moved more than skin/2 (fixed-
 * point units, minimum image) since the last one: then every pair within r_s
 * was within r_s + skin at the rebuild.  That test runs on the device and the
 * call waits for its answer.  The results therefore depend on the rebuild
 * history, not only on (positions, step).  Requires r_s + skin <= L/2.
 * skin = 0 (default) rebuilds every step by the stencil walk.  Not available
 * in batches or with rbe_adjoint (RBE_EINVAL).  Calling it again with the
 * same skin makes the next call rebuild.  rbe_get_info reports the rebuilds
 * (out[10]) and the stored-list capacity (out[11]). */
int rbe_set_verlet_skin(rbe_ctx* ctx, double skin);

/* Work decomposition of the RBL pair kernel (Sec. 2.3 stencil walk): a work
 * unit is a run of cells along x holding about atoms_per_unit atoms (0: 64;
 * shared memory caps the width); the kernel's grid has
 * ceil(units / units_per_slot) slots, one block each (0: about three units
 * per slot, and no fewer slots than one wave of resident blocks).  Results do not depend on the unit
 * width except through the order of the block partials of energies, virial
 * and net force (rounding only).  rbe_batch_autotune sets these. */
int rbe_set_rbl_tiling(rbe_ctx* ctx, int atoms_per_unit, int units_per_slot);

/* ---------------------------------------------------------------------------
 * Batched execution: many independent systems ("replicas", each its own
 * context: box, alpha, cutoffs, p, P, seed, LJ table, bonds) stepped together.
 * Every stage of the force step is one launch over all replicas, and the RBL
 * pair kernel is one persistent launch whose blocks take (replica, slot)
 * tasks from a work queue ordered by decreasing cost; one MD step is captured
 * once as a CUDA graph and replayed.  Each replica's forces, energies and
 * trajectory are bit for bit those of rbe_forces / rbe_step on its context
 * (same grids, same reduction order).
 * ------------------------------------------------------------------------- */
typedef struct rbe_batch rbe_batch;

/* A batch over nrep >= 1 distinct contexts (not owned: destroy them after
 * the batch).  All contexts must share one precision mode and have
 * debug recording off when the batch is bound. */
int rbe_batch_create(rbe_batch** out, int nrep, rbe_ctx* const* ctxs);

/* Binds replica r to n[r] atoms and its caller-owned device arrays:
 * pos[r], q[r], F[r] required; type[r], mol[r] optional (NULL); vel[r] and
 * mass[r] required by rbe_batch_step only (NULL otherwise); dt[r] and
 * accel[r] are the velocity-Verlet time step and force-to-acceleration
 * factor of replica r (may be NULL when only forces are wanted).  All
 * pointer arrays are host arrays of nrep entries.  Sets up every context for
 * its n (as rbe_forces would) and uploads the batch plan; re-bind after
 * changing a context's parameters. */
int rbe_batch_bind(rbe_batch* b, const int* n, double* const* pos, const double* const* q,
                   const int32_t* const* type, const int32_t* const* mol, double* const* F, double* const* vel,
                   const double* const* mass, const double* dt, const double* accel);

/* Forces (and each context's energies/virial/status) of every replica at MD
 * step `step`; energy may be NULL or a host array [nrep][RBE_NE] (the call
 * then waits for the stream). */
int rbe_batch_forces(rbe_batch* b, uint64_t step, double* energy, void* cuda_stream);

/* nsteps of velocity Verlet for every replica (the step of rbe_step; on
 * entry F must hold the forces at (pos, step0)), as nsteps replays of one
 * captured CUDA graph.  energy_trace: NULL or a device array
 * [nrep][nsteps][2] of (potential, kinetic / accel) per step. */
int rbe_batch_step(rbe_batch* b, uint64_t step0, int nsteps, double* energy_trace, void* cuda_stream);

/* Project-written autotuner of the pair kernel: for each family of replicas
 * (same cutoffs and p) it times the batched pair kernel over candidate
 * atoms_per_unit and units_per_slot values (coordinate descent), keeps the
 * fastest, sets them on the contexts (rbe_set_rbl_tiling), then picks the
 * kernel form (persistent blocks over the work queue, or one block per task)
 * and re-binds.  Runs force steps at step `step`: F receives the forces at
 * (pos, step); positions are not moved.  out (may be NULL, nout entries):
 * per family the chosen atoms_per_unit, units_per_slot and the kernel time
 * in ms; then the form (1 persistent, 0 one block per task), the final
 * kernel time and the untuned time (ms). */
int rbe_batch_autotune(rbe_batch* b, uint64_t step, double* out, int nout, void* cuda_stream);

/* Plan facts: out[0] replicas, [1] total atoms, [2] pair-kernel tasks,
 * [3] pair-kernel blocks, [4] its dynamic shared memory (bytes), [5] kernel
 * launches per MD step, [6] families. */
int rbe_batch_info(rbe_batch* b, double* out, int nout);

/* Waits for cuda_stream; status[r] (may be NULL) receives each replica's
 * latched status (as rbe_sync_status, which clears it); returns the first
 * non-OK status or RBE_OK. */
int rbe_batch_sync_status(rbe_batch* b, int* status, void* cuda_stream);

const char* rbe_batch_last_error(const rbe_batch* b);

/* Releases the batch (after the caller's streams are idle). */
void rbe_batch_destroy(rbe_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* RBE_H */
