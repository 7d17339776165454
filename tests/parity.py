"""Helpers shared by the GPU parity tests: run the CUDA path (through the C ABI) and the
FP64 oracle on the same seeded problem description and compare them."""
from __future__ import annotations

import numpy as np

import oracle


def rel_l2(a, b, mask=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a = a[..., mask]
        b = b[..., mask]
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def run_gpu(p, steps, precision):
    import torch
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(p, precision=precision)
    sim.set_initial()
    sim.step(steps)
    v, F, u = [t.cpu().numpy() for t in sim.fields()]
    status = sim.sync(raise_on_status=False)
    torch.cuda.synchronize()
    return sim, (v, F, u), status


def run_oracle(p, steps):
    o = oracle.Oracle(p).set_initial()
    o.step(steps)
    return o, o.fields()


def compare(p, steps, precision):
    sim, g, st = run_gpu(p, steps, precision)
    o, r = run_oracle(p, steps)
    mask = o.active_mask()
    errs = {name: rel_l2(a, b, mask) for name, a, b in zip(("v", "F", "u"), g, r)}
    # F - I relative error is the stricter measure (Eq. validation-error-measures)
    D = p.dim
    I = np.eye(D).reshape(-1)[:, None]
    gF = g[1][:, mask] - I
    rF = r[1][:, mask] - I
    errs["F-I"] = np.linalg.norm(gF - rF) / max(np.linalg.norm(rF), 1e-300)
    return errs, st, o.counts()["status"], sim, o
