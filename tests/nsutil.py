"""Helpers shared by the GPU tests (device transfer, tunes, plan comparison)."""
import numpy as np


def to_dev(A, dev):
    import torch
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).to(dev) if isinstance(v, np.ndarray) else v)
            for k, v in A.items()}


def tune_from(ns, **kw):
    t = ns.tune_default()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


from plan_checks import compare_plan, oracle_tune  # noqa: E402,F401
