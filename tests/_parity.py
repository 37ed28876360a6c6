"""Helpers for the GPU parity tests: replay the GPU's decisions in the CPU
oracle and compare."""
from __future__ import annotations

import math

import oracle


def replay(g, s, t, eps, lam, st, q_index, seed=3, tau=5, delta=0.01, peng=False, forced_lb=None):
    """Oracle GEER forced to the GPU's decisions (l_b, eta0, batches) for
    one query (stats record `st`)."""
    return oracle.geer(g, int(s), int(t), float(eps), lam, delta=delta, tau=tau, seed=seed, q_index=int(q_index),
                       forced_ell_b=int(st["ell_b"]) if forced_lb is None else forced_lb,
                       forced_eta0=int(st["eta0"]), forced_batches=int(st["batches"]), peng_ell=peng)


def compare(gpu_r, gpu_st, ref, rel_r, rel_rb):
    """Assert parity of one query: identical walks (count, steps, endpoint
    checksum), r_b and r within the relative tolerances."""
    assert gpu_st["ell"] == ref.ell
    assert gpu_st["ell_b"] == ref.ell_b
    assert gpu_st["walks"] == ref.amc.walks
    assert gpu_st["walk_steps"] == ref.amc.walk_steps
    assert int(gpu_st["checksum"]) == int(ref.amc.checksum), "walk endpoints differ"
    assert abs(gpu_st["r_b"] - ref.r_b) <= rel_rb * abs(ref.r_b), (gpu_st["r_b"], ref.r_b)
    assert abs(gpu_r - ref.r) <= rel_r * abs(ref.r), (gpu_r, ref.r)


def decisions_agree(gpu_st, ref, tau=5) -> dict:
    """Whether the oracle, free-running on its own FP64 values, would take
    the same three decisions as the GPU did."""
    smm = ref.ell == 0 or ref.free_ell_b == ref.ell_b
    if ref.amc.walks == 0:
        return {"smm": smm, "eta0": True, "stop": True}
    eta0 = int(gpu_st["eta0"]) == max(1, math.ceil(ref.amc.eta_star / 2 ** (tau - 1)))
    fb = ref.amc.free_batches
    stop = (fb == int(gpu_st["batches"])) or (fb == 0 and int(gpu_st["batches"]) == tau)
    return {"smm": smm, "eta0": eta0, "stop": stop}
