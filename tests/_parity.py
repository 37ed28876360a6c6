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


def _close(a, b, rel, absolute=0.0):
    return abs(a - b) <= rel * abs(b) + absolute


def compare(gpu_r, gpu_st, ref, rel_r, rel_rb, tau=5):
    """Assert parity of one query: identical walks (count, steps, endpoint
    checksum), r_b and r within the relative tolerances, and the switch and
    stopping quantities: psi (Eq. 9) at the switch, Eq. (17)'s volume and
    h(l - l_b), and the last batch's Bernstein error f (Eq. 7).

    psi and f carry the vectors' precision: psi within 1e-12 (FP64 path) or
    1e-6 (FP32 vectors: maxima rounded to FP32, relative 6e-8) and f within
    1e-7 or 1e-3 (its variance term is a difference of two sums, E[Z^2] - Z^2,
    so the relative error of the vectors grows by E[Z^2] / var). h is a whole
    number of walks: equal, or one ceiling step (2^tau - 1) apart when eta* /
    2^(tau-1) lies within rounding of an integer (a knife edge, counted by
    decisions_agree)."""
    fp64 = rel_r <= 1e-8
    rel_psi, rel_f = (1e-12, 1e-7) if fp64 else (1e-6, 1e-3)
    assert gpu_st["ell"] == ref.ell
    assert gpu_st["ell_b"] == ref.ell_b
    assert gpu_st["walks"] == ref.amc.walks
    assert gpu_st["walk_steps"] == ref.amc.walk_steps
    assert int(gpu_st["checksum"]) == int(ref.amc.checksum), "walk endpoints differ"
    assert abs(gpu_st["r_b"] - ref.r_b) <= rel_rb * abs(ref.r_b), (gpu_st["r_b"], ref.r_b)
    assert abs(gpu_r - ref.r) <= rel_r * abs(ref.r), (gpu_r, ref.r)
    lf = int(ref.ell) - int(ref.ell_b)
    if lf > 0:
        assert _close(float(gpu_st["psi"]), ref.amc.psi, rel_psi), ("psi", float(gpu_st["psi"]), ref.amc.psi)
        step = 2 ** tau - 1
        assert float(gpu_st["h"]) == step * int(gpu_st["eta0"]), ("h", float(gpu_st["h"]), int(gpu_st["eta0"]))
        h_ref = step * max(1, math.ceil(ref.amc.eta_star / 2 ** (tau - 1)))
        assert abs(float(gpu_st["h"]) - h_ref) <= step, ("h", float(gpu_st["h"]), h_ref)
        assert _close(float(gpu_st["f_last"]), ref.amc.f_last, rel_f, 1e-300), \
            ("f_last", float(gpu_st["f_last"]), ref.amc.f_last)
    else:
        assert float(gpu_st["psi"]) == 0.0 and float(gpu_st["h"]) == 0.0
    if int(ref.ell_b) >= 1:
        # Eq. (17)'s volume at the switch (a sum of degrees: exact)
        assert float(gpu_st["volume"]) == ref.volume, ("volume", float(gpu_st["volume"]), ref.volume)
        if lf > 0:
            assert abs(ref.h - h_ref) <= step  # the oracle's own h at the switch, same quantity


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
