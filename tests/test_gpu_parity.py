"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs and the same Philox draws.

Bars: lists, shell batches and k samples bit-exact; FP64 forces within 1e-11
per component relative to the component's condition scale A (the sum of the
absolute values of its summands, see gpu_util.cond_err): the RBE terms of
small |k| carry the weight S/P and are far larger than the net force, and a
phase k.r of size |theta| carries a rounding of order 2^-53 |theta| on either
side; energies within 1e-12 relative (E_k: relative to its condition scale);
the mixed path's force RMS error against the FP64 path at most 1e-4 relative.
"""
import numpy as np
import pytest

from gpu_util import cond_err, ek_scale, gpu_forces, literal_stats, oracle, params, rbe, rms_rel, systems, to_dev

pytestmark = pytest.mark.gpu

F_TOL = 1e-11
E_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2204_13595_gb300 import build
    build.build()
    oracle.build()


SYSTEMS = {
    "electrolyte_2000": lambda: systems.electrolyte(),
    "water_1002_wrapping_stencil": lambda: systems.water(334, seed=6),
    "water_12k": lambda: systems.water(4000, seed=4),
}


@pytest.fixture(scope="module", params=list(SYSTEMS))
def case(request):
    s = SYSTEMS[request.param]()
    step = 7
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), step)
    cap = 256
    ol = oracle.lists(s.pos, params(s), step, cap_core=cap)
    return request.param, s, step, ref, ol, cap


@pytest.mark.parametrize("precision", [rbe.FP64, rbe.MIXED])
def test_lists_and_batches_bit_exact(case, precision):
    """Both precisions decide membership by the exact rule (the mixed pair
    kernel classifies two atoms per warp pass against the union of their
    stencil rows, with the shell kept as ballot words)."""
    name, s, step, ref, ol, cap = case
    out = gpu_forces(s, step, debug_cap=cap, precision=precision)
    assert out["status"] == 0
    L = out["lists"]
    assert (L["n_core"] == ol["n_core"]).all()
    assert (L["n_shell"] == ol["n_shell"]).all()
    assert (L["core"] == ol["core"]).all()          # canonical order, -1 padded
    assert (L["batch"] == ol["batch"]).all()        # slot order


def test_k_samples_bit_exact_and_rho(case):
    name, s, step, ref, ol, cap = case
    out = gpu_forces(s, step)
    assert (out["m"] == ref["m"]).all()
    scale = np.abs(s.q).sum()
    assert np.max(np.abs(out["rho"] - ref["rho"])) < 1e-13 * scale


def test_fp64_forces_energy_virial(case):
    name, s, step, ref, ol, cap = case
    out = gpu_forces(s, step)
    assert out["status"] == 0
    ef = cond_err(out["F"], ref)
    erel = np.abs(out["E"] - ref["E"])[:5] / np.maximum(np.abs(ref["E"][:5]), 1e-300)
    ek = abs(out["E"][1] - ref["E"][1]) / ek_scale(s, ref)
    print(f"{name}: FP64 force cond err {ef:.3e}; energy rel err {erel}; E_k cond err {ek:.3e}; "
          f"E_k plain rel err {abs(out['E'][1] - ref['E'][1]) / abs(ref['E'][1]):.3e}")
    st = literal_stats(out["F"], ref)
    print(f"{name}: plain |dF|/|F| quantiles 50/90/99/99.9/max {st['rel_q']}; A/|F| quantiles {st['cond_q']}; "
          f"fraction within 1e-11 {st['frac_within_1e-11']:.6f}")
    assert ef < F_TOL
    for k in (0, 2, 3, 4):
        assert erel[k] < E_TOL, k
    assert ek < E_TOL
    assert np.allclose(out["W"], ref["W"], rtol=1e-11, atol=1e-11 * np.abs(ref["W"]).max())


def test_mixed_precision_error(case):
    name, s, step, ref, ol, cap = case
    f64 = gpu_forces(s, step)
    mix = gpu_forces(s, step, precision=rbe.MIXED)
    assert mix["status"] == 0
    e_gpu = rms_rel(mix["F"], f64["F"])
    e_orc = rms_rel(mix["F"], ref["F"])
    print(f"{name}: mixed force RMS rel err vs FP64 GPU {e_gpu:.3e}, vs oracle {e_orc:.3e}")
    assert e_gpu <= 1e-4 and e_orc <= 1e-4
    tot = np.abs(ref["E"]).sum()
    assert abs(mix["E"].sum() - ref["E"].sum()) < 1e-5 * tot


def test_deterministic_and_host_pointer_path(case):
    name, s, step, ref, ol, cap = case
    a = gpu_forces(s, step)
    b = gpu_forces(s, step, ctx=a["ctx"])
    assert (a["F"] == b["F"]).all() and (a["E"] == b["E"]).all()
    # host buffers through the same entry point (library stages the copies)
    ctx = a["ctx"]
    F = np.zeros_like(s.pos)
    E = np.zeros(rbe.NE)
    W = np.zeros(rbe.NW)
    typ = np.ascontiguousarray(s.type, np.int32)
    mol = None if s.mol is None else np.ascontiguousarray(s.mol, np.int32)
    ctx.forces(step, np.ascontiguousarray(s.pos), np.ascontiguousarray(s.q), typ, mol, F, E, W)
    assert (F == a["F"]).all() and (E == a["E"]).all() and (W == a["W"]).all()


def test_batch_covers_shell_reduces_to_truncated_sum():
    """p >= max N_S: real space equals the plain truncated sum (Eq. (2.11), N_S/p -> 1)."""
    s = systems.electrolyte()
    out = gpu_forces(s, 3, p=400)
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s, p=400), 3)
    assert cond_err(out["F"], ref) < F_TOL
    ex = oracle.ewald_exact(s.pos, s.q, s.type, s.mol, params(s, p=400), s.r_s, 0)
    assert out["E"][0] == pytest.approx(ex["E"][0], rel=1e-12)
    assert out["E"][3] == pytest.approx(ex["E"][3], rel=1e-12)


@pytest.mark.parametrize("p,P", [(1, 1), (40, 300), (33, 1025), (100, 64)])
def test_batch_size_edges(p, P):
    """p above one warp, P above one block, single samples."""
    s = systems.water(334, seed=9)
    out = gpu_forces(s, 2, p=p, P=P, debug_cap=200)
    pr = params(s, p=p, P=P)
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 2)
    ol = oracle.lists(s.pos, pr, 2, cap_core=200)
    assert (out["lists"]["batch"] == ol["batch"]).all()
    assert (out["m"] == ref["m"]).all()
    assert cond_err(out["F"], ref) < F_TOL


def test_null_type_and_mol():
    s = systems.electrolyte(n=500, L=12.6, seed=3)
    out = gpu_forces(s, 1, with_type=False)
    ref = oracle.rbe_forces(s.pos, s.q, np.zeros(s.n, np.int32), None, params(s), 1)
    assert cond_err(out["F"], ref) < F_TOL


def test_unwrapped_positions_are_wrapped():
    s = systems.electrolyte(n=500, L=12.6, seed=3)
    shift = np.random.default_rng(0).integers(-3, 4, s.pos.shape) * s.L
    out = gpu_forces(s, 1)
    s2 = systems.electrolyte(n=500, L=12.6, seed=3)
    s2.pos = s.pos + shift
    out2 = gpu_forces(s2, 1, debug_cap=64)
    ol = oracle.lists(s.pos, params(s), 1, cap_core=64)
    assert (out2["lists"]["batch"] == ol["batch"]).all()
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), 1)
    assert np.max(np.abs(out2["F"] - out["F"]) / ref["F_abs"]) < F_TOL


def test_status_errors_without_faults():
    """Input errors are reported through the status word (no device fault)."""
    s = systems.electrolyte(n=500, L=12.6, seed=3)
    s.pos[7] = s.pos[3]                      # overlapping pair
    assert gpu_forces(s, 0)["status"] == rbe.EOVERLAP
    s = systems.electrolyte(n=500, L=12.6, seed=3)
    s.q = s.q.copy()
    s.q[0] += 0.5                            # net charge
    assert gpu_forces(s, 0)["status"] == rbe.ENONNEUTRAL
    s = systems.electrolyte(n=500, L=12.6, seed=3)
    ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, 1, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    ctx.set_capacity(32, 32)                 # shell lists are ~115 long
    assert gpu_forces(s, 0, ctx=ctx)["status"] == rbe.ECAPACITY
    s = systems.electrolyte(n=500, L=12.6, seed=3)
    s.pos[11, 1] = np.nan
    assert gpu_forces(s, 0)["status"] == rbe.ENONFINITE


def test_nonfinite_input_is_reported_and_the_context_recovers():
    """All positions non-finite: RBE_ENONFINITE is latched and the atoms are
    placed on a lattice at the system's density for the rest of the step (not
    piled into one cell); after the status is read, the next step on the same
    context matches the oracle."""
    s = systems.water(4000, seed=4)
    ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    bad = systems.water(4000, seed=4)
    bad.pos = np.full_like(s.pos, np.nan)
    assert gpu_forces(bad, 1, ctx=ctx)["status"] == rbe.ENONFINITE
    out = gpu_forces(s, 2, ctx=ctx)
    assert out["status"] == 0
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), 2)
    assert cond_err(out["F"], ref) < F_TOL


@pytest.mark.parametrize("precision", [rbe.FP64, rbe.MIXED])
def test_lists_exact_at_the_radii(precision):
    """Pairs placed within 1e-9..1e-5 (relative) of r_c and r_s, in large and
    small boxes: the FP32 prefilter of the list kernel must defer to the exact
    fixed-point rule there, so the lists stay bit-exact."""
    rng = np.random.default_rng(17)
    for L, n_bg in ((20.0, 1500), (57.3, 6000)):
        s = systems.electrolyte(n=2, L=L, seed=1)
        base = rng.random((n_bg, 3)) * L
        extra = []
        for r0 in (s.r_c, s.r_s):
            for d in (-1e-5, -1e-7, -1e-9, 0.0, 1e-9, 1e-7, 1e-5):
                for _ in range(8):
                    a = rng.random(3) * L
                    u = rng.normal(size=3)
                    u /= np.linalg.norm(u)
                    extra += [a, a + r0 * (1 + d) * u]
        pos = np.concatenate([base, np.array(extra)]) % L
        n = len(pos) - len(pos) % 2
        s.pos = pos[:n]
        s.q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
        s.type = np.zeros(n, np.int32)
        s.mass = np.ones(n)
        out = gpu_forces(s, 5, debug_cap=128, precision=precision)
        ol = oracle.lists(s.pos, params(s), 5, cap_core=128)
        assert (out["lists"]["n_core"] == ol["n_core"]).all()
        assert (out["lists"]["n_shell"] == ol["n_shell"]).all()
        assert (out["lists"]["core"] == ol["core"]).all()
        assert (out["lists"]["batch"] == ol["batch"]).all()


def test_mixed_pair_energy_within_erfc_error_bound():
    """The mixed pair kernel evaluates erfc by Hastings' approximation
    (Abramowitz & Stegun 7.1.26, absolute error below 1.5e-7).  One +1/-1
    pair per system at 64 distances from 0.3 to r_s: the mixed real-space
    Coulomb energy must equal k_e q_i q_j erfc(sqrt(alpha) r)/r (math.erfc)
    within k_e |q_i q_j| / r times that bound plus FP32 rounding."""
    import math

    import torch
    s0 = systems.electrolyte(n=2, L=20.0, seed=1)
    worst = 0.0
    for r in np.linspace(0.3, s0.r_s * 0.999, 64):
        s = systems.electrolyte(n=2, L=20.0, seed=1)
        s.pos = np.array([[3.0, 4.0, 5.0], [3.0 + r * 0.6, 4.0 + r * 0.8, 5.0]])
        s.q = np.array([1.0, -1.0])
        s.type = np.zeros(2, np.int32)
        out = gpu_forces(s, 1, precision=rbe.MIXED)
        assert out["status"] == 0
        exact = s.k_e * s.q[0] * s.q[1] * math.erfc(math.sqrt(s.alpha) * r) / r
        bound = s.k_e / r * 1.5e-7 + 4e-7 * abs(exact) + 1e-12
        err = abs(out["E"][rbe.E_REAL] - exact)
        worst = max(worst, err / bound)
        assert err <= bound, (r, err, bound)
    print(f"mixed pair energy: worst error / bound {worst:.3f}")


def test_fp64_pair_energy_matches_erfc():
    """The FP64 pair kernel evaluates erfc and erf by W. J. Cody's rational
    Chebyshev approximations (Math. Comp. 23, 1969) from the e^{-x^2} of the
    force term.  One +1/-1 pair per system at 64 distances from 0.3 to r_s,
    once as an ordinary pair and once as a same-molecule (excluded) pair:
    the FP64 real-space energy must equal k_e q_i q_j erfc(sqrt(alpha) r)/r
    (math.erfc), and the exclusion energy -k_e q_i q_j erf(sqrt(alpha) r)/r
    (math.erf), within 5e-15 relative plus the condition number of the
    function (1 + 2 x^2 for erfc, at most 1 for erf) times the relative
    error of the distance itself (the wrapped FP64 positions carry a few ulp
    of coordinates up to 12 A); the arguments cover all three of Cody's
    intervals (x = sqrt(alpha) r up to 6.1 with alpha = 1.5)."""
    import math
    worst = 0.0
    for alpha in (None, 1.5):
        for r in np.linspace(0.3, systems.electrolyte(n=2, L=20.0, seed=1).r_s * 0.999, 64):
            for excl in (False, True):
                s = systems.electrolyte(n=2, L=20.0, seed=1)
                if alpha is not None:
                    s.alpha = alpha
                s.pos = np.array([[3.0, 4.0, 5.0], [3.0 + r * 0.6, 4.0 + r * 0.8, 5.0]])
                s.q = np.array([1.0, -1.0])
                s.type = np.zeros(2, np.int32)
                s.mol = np.array([0, 0], np.int32) if excl else None
                out = gpu_forces(s, 1, precision=rbe.FP64)
                assert out["status"] == 0
                x = math.sqrt(s.alpha) * r
                if excl:
                    exact, got = -s.k_e * s.q[0] * s.q[1] * math.erf(x) / r, out["E"][rbe.E_EXCL]
                else:
                    exact, got = s.k_e * s.q[0] * s.q[1] * math.erfc(x) / r, out["E"][rbe.E_REAL]
                rel = abs(got - exact) / abs(exact)
                cond = 1.0 if excl else 1.0 + 2.0 * x * x
                bound = 5e-15 + cond * (4e-16 + 6e-15 / r)
                worst = max(worst, rel / bound)
                assert rel < bound, (alpha, r, excl, rel, bound)
    print(f"FP64 pair energy: worst relative error / bound {worst:.3f}")
