// rbe_batch.cu -- host side of batched execution (rbe_batch_* in include/rbe.h).
//
// Many independent systems ("replicas") step together.  Every replica keeps
// its own context; the plan built here gives each stage of the force step
// (Algorithm 1, force steps) one launch over all replicas:
//   cells:   zero counts, quantise+count, scan (block per replica), scatter,
//            in-cell sort, gather
//   k space: sample, rho partials, rho sum, [bonded water]
//   pairs:   one launch of the RBL kernel over all (replica, slot) tasks,
//            ordered by decreasing estimated cost: persistent resident
//            blocks pulling tasks from a device queue, or one block per task
//            (the autotuner picks the faster form)
//   finish:  finalize (block per replica), k-space force + combination
// and one MD step (velocity Verlet around it) is captured once as a CUDA
// graph and replayed, the step number living in a device control block.
// Each replica's blocks see the same block indices and grid sizes as in its
// single-system launches, so the two paths give identical bits.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rbe_internal.cuh"

struct rbe_batch {
    int nrep = 0;
    std::vector<rbe_ctx*> ctx;
    // bound arrays (for re-binding after tuning)
    std::vector<int> n;
    std::vector<double*> pos, F, vel;
    std::vector<const double*> q, mass;
    std::vector<const int32_t*> type, mol;
    std::vector<double> dt, accel;
    bool bound = false, can_step = false;
    // plan
    std::vector<RepDev> rep;
    std::vector<unsigned char> rbl_args;
    std::vector<int> family;
    int nfam = 0;
    RepDev* d_rep = nullptr;
    unsigned char* d_rbl = nullptr;
    int* d_off = nullptr;
    int2* d_tasks = nullptr;
    size_t tasks_cap = 0;
    BatchCtl* d_ctl = nullptr;
    int* d_mask = nullptr;   // replicas whose Langevin force is made at entry
    BatchPlan plan{};
    int persistent = 1;      // pair kernel form (autotuned)
    bool lang = false;       // some replica runs the Langevin thermostat
    int launches_force = 0, launches_step = 0;
    long total_atoms = 0;
    int n_sm = 0;
    // one MD step as a CUDA graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    char err[512] = {0};
};

namespace {

int berr(rbe_batch* b, int code, const char* fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define BATCH_TRY(b, call)                                                                           \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return berr(b, RBE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool on_device(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void drop_graph(rbe_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

void free_plan(rbe_batch* b)
{
    drop_graph(b);
    void* ptrs[] = {b->d_rep, b->d_rbl, b->d_off, b->d_tasks, b->d_ctl, b->d_mask};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    b->d_rep = nullptr; b->d_rbl = nullptr; b->d_off = nullptr; b->d_tasks = nullptr; b->d_ctl = nullptr;
    b->d_mask = nullptr;
    b->tasks_cap = 0;
}

// Families: replicas sharing cutoffs and shell batch size share a tiling.
void assign_families(rbe_batch* b)
{
    b->family.assign(b->nrep, -1);
    std::vector<int> head;
    for (int r = 0; r < b->nrep; ++r) {
        const RbeConsts& c = b->ctx[r]->c;
        for (size_t f = 0; f < head.size(); ++f) {
            const RbeConsts& h = b->ctx[head[f]]->c;
            if (h.r_c == c.r_c && h.r_s == c.r_s && h.p == c.p) { b->family[r] = (int)f; break; }
        }
        if (b->family[r] < 0) {
            b->family[r] = (int)head.size();
            head.push_back(r);
        }
    }
    b->nfam = (int)head.size();
}

int ceil_div(long a, long d) { return (int)((a + d - 1) / d); }

// Builds and uploads the plan from the bound arrays and the contexts' current
// parameters.
int build_plan(rbe_batch* b)
{
    const int nr = b->nrep;
    drop_graph(b);
    int prec = b->ctx[0]->precision;
    for (int r = 0; r < nr; ++r) {
        rbe_ctx* ctx = b->ctx[r];
        if (ctx->precision != prec) return berr(b, RBE_EINVAL, "replica %d: all replicas need one precision mode", r);
        if (ctx->debug) return berr(b, RBE_EINVAL, "replica %d: debug recording must be off in a batch", r);
        if (ctx->skin > 0.0) return berr(b, RBE_EINVAL, "replica %d: the Verlet skin is not batched", r);
        int rc = ctx_prepare(ctx, b->n[r]);
        if (rc) return berr(b, rc, "replica %d: %s", r, ctx->err);
    }
    if (b->d_ctl == nullptr) {
        BATCH_TRY(b, cudaMalloc((void**)&b->d_ctl, sizeof(BatchCtl)));
        BATCH_TRY(b, cudaMemset(b->d_ctl, 0, sizeof(BatchCtl)));
    }
    BATCH_TRY(b, cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->ctx[0]->device));

    // replica views and pair-kernel arguments
    const size_t ab = rbl_args_bytes();
    b->rep.assign(nr, RepDev{});
    b->rbl_args.assign(ab * nr, 0);
    std::vector<int> cnt[BK_COUNT];
    for (int k = 0; k < BK_COUNT; ++k) cnt[k].assign(nr, 0);
    int rho_threads = 32, smem = 0;
    b->total_atoms = 0;
    bool bonds = false, lang = false;
    struct Task { double cost; int r, s; };
    std::vector<Task> tasks;
    for (int r = 0; r < nr; ++r) {
        rbe_ctx* ctx = b->ctx[r];
        const int n = b->n[r];
        RepDev& d = b->rep[r];
        d.n = n;
        d.nmol = ctx->n_wmol;
        d.n_bonded_atoms = ctx->n_wmol > 0 ? 3 * ctx->n_wmol : 0;
        d.ncells = ctx->ncells;
        d.grid_q = ctx->grid_q;
        d.grid_rho = ctx->grid_rho;
        d.grid_rbl = ctx->grid_rbl;
        d.grid_bond = ctx->n_wmol > 0 ? ctx->grid_bond : 0;
        d.rho_chunk = (n + ctx->grid_rho - 1) / ctx->grid_rho;
        d.kb = ctx->kb; d.r0 = ctx->r0; d.kth = ctx->kth; d.th0 = ctx->th0;
        d.dt = b->dt.empty() ? 0.0 : b->dt[r];
        d.accel = b->accel.empty() ? 1.0 : b->accel[r];
        d.c = ctx->c;
        d.pos = b->pos[r]; d.vel = b->vel[r]; d.mass = b->mass[r]; d.q = b->q[r];
        d.type = b->type[r]; d.mol = b->mol[r]; d.F = b->F[r];
        d.cell_count = ctx->cell_count; d.cell_start = ctx->cell_start; d.cell_of = ctx->cell_of;
        d.slot = ctx->slot; d.perm = ctx->perm; d.sx_of = ctx->sx_of; d.skey = ctx->skey;
        d.s4 = ctx->s4; d.f4 = ctx->f4; d.p4 = ctx->p4; d.tm = ctx->tm;
        d.rec_s4 = ctx->rec_s4; d.rec_p4 = ctx->rec_p4; d.rec_tm = ctx->rec_tm;
        d.part_q = ctx->part_q; d.part_rbl = ctx->part_rbl; d.part_bond = ctx->part_bond; d.ke_part = ctx->ke_part;
        d.kT = ctx->kT; d.km = ctx->km; d.kv = ctx->kv; d.rho_part = ctx->rho_part; d.rho = ctx->rho;
        d.totals = ctx->totals; d.F_real = ctx->F_real; d.F_bond = ctx->F_bond; d.status = ctx->status;
        d.kpool = ctx->kpool_buf;
        d.cis = ctx->cis;
        d.FL = nullptr;
        d.lang_c1 = d.lang_c2 = 0.0;
        if (ctx->lang_tau > 0.0 && b->can_step) {
            int rc = ctx_grow_lang(ctx, n);
            if (rc) return berr(b, rc, "replica %d: %s", r, ctx->err);
            d.FL = ctx->F_lang;
            d.lang_c1 = d.accel * ctx->lang_tau;
            d.lang_c2 = 24.0 * ctx->lang_kT / (d.lang_c1 * d.dt);
            lang = true;
        }
        rbl_fill_args(ctx, n, b->rbl_args.data() + ab * r);

        cnt[BK_CELLS][r] = ceil_div(ctx->ncells + 1, 256);
        cnt[BK_ATOMS][r] = ceil_div(n, 256);
        cnt[BK_Q][r] = ctx->grid_q;
        cnt[BK_KS][r] = ceil_div(ctx->c.P, 256);
        cnt[BK_RHO][r] = ctx->grid_rho;
        cnt[BK_BOND][r] = d.grid_bond;
        cnt[BK_REP][r] = 1;
        cnt[BK_RS][r] = ceil_div(ctx->c.P, 8);         // rho sum: one warp per k
        if (d.grid_bond > 0) bonds = true;
        const int P = ctx->c.P;
        const int th = ((P < 1024 ? P : 1024) + 31) / 32 * 32;
        rho_threads = th > rho_threads ? th : rho_threads;
        const int sm = rbl_smem_bytes(ctx);
        smem = sm > smem ? sm : smem;
        b->total_atoms += n;

        // task cost: atoms of the slot x (candidates classified + pair terms)
        const double PI = 3.14159265358979323846;
        const double rho_n = (double)n / (ctx->c.L * ctx->c.L * ctx->c.L);
        const double rc3 = ctx->c.r_c * ctx->c.r_c * ctx->c.r_c, rs3 = ctx->c.r_s * ctx->c.r_s * ctx->c.r_s;
        const double mc = 4.0 / 3.0 * PI * rc3 * rho_n, ms = 4.0 / 3.0 * PI * (rs3 - rc3) * rho_n;
        const double per_atom = 3.0 * (mc + ms) + 4.0 * (mc + (ms < ctx->c.p ? ms : ctx->c.p));
        const long units = rbl_units(ctx);
        const double apu = (double)n / (double)units;
        for (int s = 0; s < ctx->grid_rbl; ++s) {
            const long us = (units - 1 - s) / ctx->grid_rbl + 1;
            tasks.push_back(Task{(double)us * apu * per_atom, r, s});
        }
    }
    std::stable_sort(tasks.begin(), tasks.end(), [](const Task& x, const Task& y) { return x.cost > y.cost; });

    // block offsets of every stage
    std::vector<int> off((size_t)BK_COUNT * (nr + 1));
    for (int k = 0; k < BK_COUNT; ++k) {
        int acc = 0;
        for (int r = 0; r < nr; ++r) {
            off[(size_t)k * (nr + 1) + r] = acc;
            acc += cnt[k][r];
        }
        off[(size_t)k * (nr + 1) + nr] = acc;
        b->plan.total[k] = acc;
    }

    int bps = rbl_max_blocks_per_sm(prec, smem);
    if (bps < 1) return berr(b, RBE_ECAPACITY, "batched pair kernel does not fit: %d bytes of shared memory", smem);

    // upload
    if (!b->d_rep) {
        BATCH_TRY(b, cudaMalloc((void**)&b->d_rep, sizeof(RepDev) * nr));
        BATCH_TRY(b, cudaMalloc((void**)&b->d_rbl, ab * nr));
        BATCH_TRY(b, cudaMalloc((void**)&b->d_off, sizeof(int) * off.size()));
    }
    if (tasks.size() > b->tasks_cap) {
        if (b->d_tasks) cudaFree(b->d_tasks);
        b->d_tasks = nullptr;
        BATCH_TRY(b, cudaMalloc((void**)&b->d_tasks, sizeof(int2) * tasks.size()));
        b->tasks_cap = tasks.size();
    }
    std::vector<int2> ht(tasks.size());
    for (size_t t = 0; t < tasks.size(); ++t) ht[t] = make_int2(tasks[t].r, tasks[t].s);
    BATCH_TRY(b, cudaMemcpy(b->d_rep, b->rep.data(), sizeof(RepDev) * nr, cudaMemcpyHostToDevice));
    BATCH_TRY(b, cudaMemcpy(b->d_rbl, b->rbl_args.data(), ab * nr, cudaMemcpyHostToDevice));
    BATCH_TRY(b, cudaMemcpy(b->d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    BATCH_TRY(b, cudaMemcpy(b->d_tasks, ht.data(), sizeof(int2) * ht.size(), cudaMemcpyHostToDevice));

    BatchPlan& p = b->plan;
    p.nrep = nr;
    p.precision = prec;
    p.rep = b->d_rep;
    for (int k = 0; k < BK_COUNT; ++k) p.off[k] = b->d_off + (size_t)k * (nr + 1);
    p.ctl = b->d_ctl;
    p.rho_threads = rho_threads;
    p.rbl_args = b->d_rbl;
    p.tasks = b->d_tasks;
    p.ntasks = (int)tasks.size();
    p.rbl_grid = bps * b->n_sm;
    p.rbl_smem = smem;
    p.rbl_persistent = b->persistent;
    b->launches_force = 6 + 3 + (bonds ? 1 : 0) + 1 + 2;
    // + control, two half kicks, kinetic energy + trace, Langevin force
    b->launches_step = b->launches_force + 1 + 2 + 2 + (lang ? 1 : 0);
    b->lang = lang;
    return RBE_OK;
}

void enqueue_forces(const BatchPlan& p, cudaStream_t st)
{
    launch_cells_batch(p, st);
    launch_kspace_pre_batch(p, st);
    launch_rbl_batch(p, st);
    launch_kspace_post_batch(p, st);
}

int launch_status(rbe_batch* b)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return berr(b, RBE_ECUDA, "batched launch failed: %s", cudaGetErrorString(e));
    return RBE_OK;
}

int ensure_graph(rbe_batch* b)
{
    if (b->exec) return RBE_OK;
    if (!b->cap_stream) BATCH_TRY(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    BATCH_TRY(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const BatchPlan& p = b->plan;
    launch_vv_batch(p, 1, b->cap_stream);
    launch_ctl_batch(p, 1, 0, nullptr, 0, b->cap_stream);
    enqueue_forces(p, b->cap_stream);
    if (b->lang) launch_langevin_batch(p, nullptr, b->cap_stream);
    launch_vv_batch(p, 0, b->cap_stream);
    launch_ke_trace_batch(p, b->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess || !g) {
        cudaGetLastError();
        return berr(b, RBE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return berr(b, RBE_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return RBE_OK;
}

// Minimum over `reps` timed launches of the batched pair kernel (ms).
int time_pairs(rbe_batch* b, cudaStream_t st, int reps, double* ms)
{
    cudaEvent_t e0, e1;
    BATCH_TRY(b, cudaEventCreate(&e0));
    BATCH_TRY(b, cudaEventCreate(&e1));
    double best = 1e30;
    for (int k = 0; k < reps; ++k) {
        launch_ctl_batch(b->plan, 2, 0, nullptr, 0, st);
        cudaEventRecord(e0, st);
        launch_rbl_batch(b->plan, st);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return berr(b, RBE_ECUDA, "timing failed: %s", cudaGetErrorString(e));
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        best = t < best ? t : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return launch_status(b);
}

}  // namespace

extern "C" {

int rbe_batch_create(rbe_batch** out, int nrep, rbe_ctx* const* ctxs)
{
    if (!out) return RBE_EINVAL;
    *out = nullptr;
    if (nrep < 1 || !ctxs) return RBE_EINVAL;
    for (int r = 0; r < nrep; ++r) {
        if (!ctxs[r]) return RBE_EINVAL;
        for (int s = 0; s < r; ++s)
            if (ctxs[s] == ctxs[r]) return RBE_EINVAL;
    }
    rbe_batch* b = new rbe_batch();
    b->nrep = nrep;
    b->ctx.assign(ctxs, ctxs + nrep);
    assign_families(b);
    *out = b;
    return RBE_OK;
}

int rbe_batch_bind(rbe_batch* b, const int* n, double* const* pos, const double* const* q,
                   const int32_t* const* type, const int32_t* const* mol, double* const* F, double* const* vel,
                   const double* const* mass, const double* dt, const double* accel)
{
    if (!b) return RBE_EINVAL;
    if (!n || !pos || !q || !F) return berr(b, RBE_EINVAL, "n, pos, q and F are required");
    const int nr = b->nrep;
    bool step_ok = vel && mass && dt && accel;
    for (int r = 0; r < nr; ++r) {
        if (n[r] < 1 || !pos[r] || !q[r] || !F[r]) return berr(b, RBE_EINVAL, "replica %d: n, pos, q, F", r);
        if (!on_device(pos[r]) || !on_device(q[r]) || !on_device(F[r]) || (type && type[r] && !on_device(type[r])) ||
            (mol && mol[r] && !on_device(mol[r])))
            return berr(b, RBE_EINVAL, "replica %d: batched arrays must be device pointers", r);
        if (step_ok) {
            if (!vel[r] || !mass[r] || !on_device(vel[r]) || !on_device(mass[r]) || !(dt[r] > 0) || !(accel[r] > 0))
                return berr(b, RBE_EINVAL, "replica %d: vel, mass (device), dt > 0 and accel > 0", r);
        }
    }
    b->n.assign(n, n + nr);
    b->pos.assign(pos, pos + nr);
    b->q.assign(q, q + nr);
    b->F.assign(F, F + nr);
    b->type.assign(nr, nullptr);
    b->mol.assign(nr, nullptr);
    if (type) b->type.assign(type, type + nr);
    if (mol) b->mol.assign(mol, mol + nr);
    b->vel.assign(nr, nullptr);
    b->mass.assign(nr, nullptr);
    b->dt.clear();
    b->accel.clear();
    if (step_ok) {
        b->vel.assign(vel, vel + nr);
        b->mass.assign(mass, mass + nr);
        b->dt.assign(dt, dt + nr);
        b->accel.assign(accel, accel + nr);
    }
    b->can_step = step_ok;
    b->bound = false;
    int rc = build_plan(b);
    if (rc) return rc;
    b->bound = true;
    return RBE_OK;
}

int rbe_batch_forces(rbe_batch* b, uint64_t step, double* energy, void* cuda_stream)
{
    if (!b) return RBE_EINVAL;
    if (!b->bound) return berr(b, RBE_EINVAL, "batch is not bound");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    launch_ctl_batch(b->plan, 0, step, nullptr, 0, st);
    enqueue_forces(b->plan, st);
    int rc = launch_status(b);
    if (rc) return rc;
    if (energy) {
        for (int r = 0; r < b->nrep; ++r)
            BATCH_TRY(b, cudaMemcpyAsync(energy + (size_t)r * RBE_NE, b->ctx[r]->totals, sizeof(double) * RBE_NE,
                                         cudaMemcpyDefault, st));
        BATCH_TRY(b, cudaStreamSynchronize(st));
    }
    return RBE_OK;
}

int rbe_batch_step(rbe_batch* b, uint64_t step0, int nsteps, double* energy_trace, void* cuda_stream)
{
    if (!b) return RBE_EINVAL;
    if (!b->bound) return berr(b, RBE_EINVAL, "batch is not bound");
    if (!b->can_step) return berr(b, RBE_EINVAL, "bind vel, mass, dt and accel to step");
    if (nsteps < 0) return berr(b, RBE_EINVAL, "nsteps < 0");
    if (energy_trace && !on_device(energy_trace)) return berr(b, RBE_EINVAL, "energy_trace must be a device pointer");
    if (nsteps == 0) return RBE_OK;
    int rc = ensure_graph(b);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    launch_ctl_batch(b->plan, 0, step0, energy_trace, nsteps, st);
    if (b->lang) {
        // F^L at entry (step0) for the thermostatted replicas whose context does
        // not already hold it from a run that ended at step0 (as rbe_step)
        std::vector<int> mask(b->nrep, 0);
        bool any = false;
        for (int r = 0; r < b->nrep; ++r) {
            const rbe_ctx* c = b->ctx[r];
            mask[r] = (c->lang_tau > 0.0 && !(c->lang_valid && c->lang_step == step0 && c->lang_n == b->n[r])) ? 1 : 0;
            any = any || mask[r];
        }
        if (any) {
            if (!b->d_mask) BATCH_TRY(b, cudaMalloc((void**)&b->d_mask, sizeof(int) * b->nrep));
            BATCH_TRY(b, cudaMemcpyAsync(b->d_mask, mask.data(), sizeof(int) * b->nrep, cudaMemcpyHostToDevice, st));
            BATCH_TRY(b, cudaStreamSynchronize(st));      // mask is host memory of this call
            launch_langevin_batch(b->plan, b->d_mask, st);
        }
    }
    for (int k = 0; k < nsteps; ++k) BATCH_TRY(b, cudaGraphLaunch(b->exec, st));
    if (b->lang)
        for (int r = 0; r < b->nrep; ++r) {
            rbe_ctx* c = b->ctx[r];
            if (c->lang_tau > 0.0) { c->lang_step = step0 + (uint64_t)nsteps; c->lang_valid = 1; c->lang_n = b->n[r]; }
        }
    return launch_status(b);
}

int rbe_batch_autotune(rbe_batch* b, uint64_t step, double* out, int nout, void* cuda_stream)
{
    if (!b) return RBE_EINVAL;
    if (!b->bound) return berr(b, RBE_EINVAL, "batch is not bound");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nr = b->nrep;
    // sorted arrays and k samples at `step` (the tiling does not change them)
    launch_ctl_batch(b->plan, 0, step, nullptr, 0, st);
    enqueue_forces(b->plan, st);
    int rc = launch_status(b);
    if (rc) return rc;
    BATCH_TRY(b, cudaStreamSynchronize(st));

    auto apply = [&](int fam, int a, int u) {
        for (int r = 0; r < nr; ++r)
            if (b->family[r] == fam) rbe_set_rbl_tiling(b->ctx[r], a, u);
    };
    auto measure = [&](double* ms) -> int {
        int rc2 = build_plan(b);
        if (rc2) return rc2;
        return time_pairs(b, st, 3, ms);
    };
    double t_untuned = 0.0;
    for (int f = 0; f < b->nfam; ++f) apply(f, 0, 0);
    if ((rc = measure(&t_untuned))) return rc;

    static const int cand_apu[] = {16, 24, 32, 48, 64, 96, 128};
    static const int cand_ups[] = {0, 1, 2, 3, 4, 8};
    std::vector<double> res;
    double best_all = t_untuned;
    for (int f = 0; f < b->nfam; ++f) {
        int best_a = 0, best_u = 0;
        double best = best_all;
        for (int a : cand_apu) {
            apply(f, a, best_u);
            double t = 0.0;
            if ((rc = measure(&t))) return rc;
            if (t < best) { best = t; best_a = a; }
        }
        for (int u : cand_ups) {
            apply(f, best_a, u);
            double t = 0.0;
            if ((rc = measure(&t))) return rc;
            if (t < best) { best = t; best_u = u; }
        }
        apply(f, best_a, best_u);
        best_all = best;
        res.push_back(best_a);
        res.push_back(best_u);
        res.push_back(best);
    }
    // kernel form: persistent blocks over the queue, or one block per task
    {
        const int cur = b->persistent;
        b->persistent = 1 - cur;
        double t = 0.0;
        if ((rc = measure(&t))) return rc;
        if (!(t < best_all)) b->persistent = cur;
        else best_all = t;
    }
    res.push_back((double)b->persistent);
    res.push_back(best_all);
    res.push_back(t_untuned);
    if ((rc = build_plan(b))) return rc;
    // leave the forces at `step` consistent with the chosen tiling
    launch_ctl_batch(b->plan, 0, step, nullptr, 0, st);
    enqueue_forces(b->plan, st);
    if ((rc = launch_status(b))) return rc;
    BATCH_TRY(b, cudaStreamSynchronize(st));
    if (out)
        for (int k = 0; k < nout && k < (int)res.size(); ++k) out[k] = res[k];
    return RBE_OK;
}

int rbe_batch_info(rbe_batch* b, double* out, int nout)
{
    if (!b || !out) return RBE_EINVAL;
    double v[7] = {(double)b->nrep, (double)b->total_atoms, (double)b->plan.ntasks, (double)b->plan.rbl_grid,
                   (double)b->plan.rbl_smem, (double)b->launches_step, (double)b->nfam};
    for (int k = 0; k < nout && k < 7; ++k) out[k] = v[k];
    return RBE_OK;
}

int rbe_batch_sync_status(rbe_batch* b, int* status, void* cuda_stream)
{
    if (!b) return RBE_EINVAL;
    int first = RBE_OK;
    for (int r = 0; r < b->nrep; ++r) {
        int s = rbe_sync_status(b->ctx[r], cuda_stream);
        if (status) status[r] = s;
        if (s != RBE_OK && first == RBE_OK) first = s;
    }
    return first;
}

const char* rbe_batch_last_error(const rbe_batch* b) { return b ? b->err : "null batch"; }

void rbe_batch_destroy(rbe_batch* b)
{
    if (!b) return;
    free_plan(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

}  // extern "C"
