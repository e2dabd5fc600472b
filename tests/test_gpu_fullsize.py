"""Parity at the benchmark sizes (90k-atom and 1.2M-atom water), in the launch
configuration bench.py times, against the oracle run in full on the host cores."""
import numpy as np
import pytest

from gpu_util import cond_err, ek_scale, gpu_forces, literal_stats, oracle, params, rbe, rms_rel, systems

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_mol,seed", [(30000, 2), (400000, 3)])
def test_full_size_water(n_mol, seed):
    s = systems.water(n_mol, seed=seed)
    step = 11
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), step)
    f64 = gpu_forces(s, step, debug_cap=160)
    assert f64["status"] == 0
    # lists of every atom, bit for bit
    ol = oracle.lists(s.pos, params(s), step, cap_core=160)
    assert (f64["lists"]["n_core"] == ol["n_core"]).all()
    assert (f64["lists"]["n_shell"] == ol["n_shell"]).all()
    assert (f64["lists"]["core"] == ol["core"]).all()
    assert (f64["lists"]["batch"] == ol["batch"]).all()
    assert (f64["m"] == ref["m"]).all()
    ef = cond_err(f64["F"], ref)
    erel = np.abs(f64["E"] - ref["E"])[:5] / np.abs(ref["E"][:5])
    ek = abs(f64["E"][1] - ref["E"][1]) / ek_scale(s, ref)
    print(f"water {s.n}: FP64 force cond err {ef:.3e}; energy rel err {erel}; E_k cond err {ek:.3e}; "
          f"E_k plain rel err {abs(f64['E'][1] - ref['E'][1]) / abs(ref['E'][1]):.3e}")
    st = literal_stats(f64["F"], ref)
    print(f"water {s.n}: plain |dF|/|F| quantiles 50/90/99/99.9/max {st['rel_q']}; A/|F| quantiles "
          f"{st['cond_q']}; fraction within 1e-11 {st['frac_within_1e-11']:.6f}")
    assert ef < 1e-11
    for k in (0, 2, 3, 4):
        assert erel[k] < 1e-12, k
    assert ek < 1e-12
    mix = gpu_forces(s, step, precision=rbe.MIXED, debug_cap=160)
    assert mix["status"] == 0
    for k in ("n_core", "n_shell", "core", "batch"):
        assert (mix["lists"][k] == ol[k]).all(), k
    em = rms_rel(mix["F"], f64["F"])
    print(f"water {s.n}: mixed force RMS rel err vs FP64 {em:.3e}")
    assert em <= 1e-4
