"""Helpers shared by the GPU tests (device transfer, plan comparison)."""
import numpy as np

import oracle


def to_dev(A, dev):
    import torch
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).to(dev) if isinstance(v, np.ndarray) else v)
            for k, v in A.items()}


def tune_from(ns, **kw):
    t = ns.tune_default()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def oracle_tune(t):
    d = t.as_dict()
    d.pop("l2_hints")
    d.pop("TN")
    return d


def compare_plan(plan, ref):
    """Every plan array bit-exact against the CPU reference partition."""
    st = plan.stats()
    for k in oracle.PLAN_SCALARS:
        assert st[k] == ref[k], f"scalar {k}: device {st[k]} vs reference {ref[k]}"
    for name in oracle.PLAN_ARRAYS:
        got = plan.export(name)
        exp = np.asarray(ref[name])
        if name in ("win_dptr",) and ref["n_win"] == 0:
            continue
        assert got.dtype == exp.dtype, (name, got.dtype, exp.dtype)
        assert got.shape == exp.shape, (name, got.shape, exp.shape)
        if not np.array_equal(got.view(np.uint8), exp.view(np.uint8)):
            bad = np.nonzero(got != exp)[0][:10]
            raise AssertionError(f"plan array {name} differs at {bad}: {got[bad]} vs {exp[bad]}")
