"""rbe_forces with host inputs (include/rbe.h): pinned host buffers are read by
the device in place, pageable ones are copied first.  Both must give, bit for
bit, the forces and energies of the same call on device arrays (the
quantisation writes the same per-atom records whichever memory it reads), and
through them the oracle's."""
import numpy as np
import pytest

from gpu_util import cond_err, oracle, params, rbe, systems

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["electrolyte", "water"])
@pytest.mark.parametrize("precision", [rbe.FP64, rbe.MIXED])
def test_pinned_pageable_and_device_inputs_agree(kind, precision):
    import torch
    s = systems.electrolyte() if kind == "electrolyte" else systems.water(4000, seed=4)
    step = 6
    typ = s.type.astype(np.int32)
    mol = None if s.mol is None else s.mol.astype(np.int32)
    out = {}
    for where in ("device", "pageable", "pinned"):
        ctx = rbe.Context.for_system(s, precision=precision)
        if where == "device":
            t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
            args = (t(s.pos), t(s.q), t(typ, torch.int32), None if mol is None else t(mol, torch.int32))
            F = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
            E = torch.zeros(rbe.NE, dtype=torch.float64, device="cuda")
        elif where == "pageable":
            args = (s.pos.copy(), s.q.copy(), typ.copy(), None if mol is None else mol.copy())
            F = np.zeros((s.n, 3))
            E = np.zeros(rbe.NE)
        else:
            t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt).pin_memory()
            args = (t(s.pos), t(s.q), t(typ, torch.int32), None if mol is None else t(mol, torch.int32))
            F = torch.zeros((s.n, 3), dtype=torch.float64).pin_memory()
            E = torch.zeros(rbe.NE, dtype=torch.float64).pin_memory()
        ctx.forces(step, *args, F, E)
        assert ctx.sync_status() == 0, where
        to_np = lambda a: a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
        out[where] = (to_np(F).copy(), to_np(E).copy())
        ctx.close()
    for where in ("pageable", "pinned"):
        assert np.array_equal(out[where][0], out["device"][0]), where
        assert np.array_equal(out[where][1], out["device"][1]), where
    if precision == rbe.FP64:
        ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), step)
        assert cond_err(out["pinned"][0], ref) < 1e-11


def test_pinned_inputs_without_type_and_mol():
    import torch
    s = systems.electrolyte()
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    ctx = rbe.Context.for_system(s)
    F1 = torch.zeros((s.n, 3), dtype=torch.float64).pin_memory()
    ctx.forces(3, t(s.pos).pin_memory(), t(s.q).pin_memory(), None, None, F1)
    assert ctx.sync_status() == 0
    F2 = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    ctx.forces(3, t(s.pos).cuda(), t(s.q).cuda(), None, None, F2)
    assert ctx.sync_status() == 0
    assert torch.equal(F1, F2.cpu())
    ctx.close()
