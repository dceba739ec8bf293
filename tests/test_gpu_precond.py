"""The learned preconditioner against Teter's, and its automatic fallback (GPU).

The band minimiser (JDFTx paper, Sec. 2.1 Minimize) takes the network's
per-coefficient preconditioner K_theta in place of Teter's.  Teter's
preconditioner is its fallback: when the network's direction is not a finite
descent direction, gives no lower energy, or makes no progress for 40
iterations, Teter's takes over for the rest of the call (report field
precond_fallback).  Deliberately broken weights must trigger that and still
reach the exact energy.

The comparison with Teter's preconditioner records what the committed network
gains, and what it does not: with either preconditioner the mixed-precision
minimisation reaches the exact energy faster than plain FP64 + Teter, but on
a held-out cell (seed 2009, never seen in training) the network needs about
as many iterations as Teter, not fewer.
"""
import json
import os

import numpy as np
import pytest

from tests.systems import GpuSystem, OracleSystem, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_eigs.json")))


def _small():
    w = workload("small")
    o = OracleSystem(w)
    return o, GpuSystem(w, o.atoms)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("kind", ["nan", "zero_output"])
def test_broken_weights_fall_back_to_teter(kind, prec):
    from paper_1708_03621_gb300 import jdft
    if kind == "nan":
        params = np.full(jdft.MLP_NPARAM, np.nan, dtype=np.float32)
    else:
        # all weights zero, output bias -200: softplus(-200) = 0 in FP32, so K = 0 everywhere
        params = np.zeros(jdft.MLP_NPARAM, dtype=np.float32)
        params[-1] = -200.0
    m = jdft.Mlp(params)
    o, g = _small()
    C = torch.tensor(o.coeffs(16), device="cuda")
    rep = jdft.jdft_minimize_bands(g.basis, 0, C, tol=1e-8, max_iter=3000, precond="mlp", prec=prec, mlp=m)
    assert rep["converged"] and rep["precond_fallback"] == 1, rep
    assert abs(rep["energy"] - GOLDEN["E_ref"]) < 1e-6


def test_working_weights_keep_the_network():
    from paper_1708_03621_gb300 import jdft, learned
    m = jdft.Mlp(learned.load_weights())
    o, g = _small()
    C = torch.tensor(o.coeffs(16), device="cuda")
    rep = jdft.jdft_minimize_bands(g.basis, 0, C, tol=1e-8, max_iter=3000, precond="mlp", prec="bf16x3", mlp=m)
    assert rep["converged"] and rep["precond_fallback"] == 0, rep
    assert abs(rep["energy"] - GOLDEN["E_ref"]) < 1e-6


def test_mixed_learned_beats_fp64_teter_in_time_to_dE():
    """The scope's target on the 48^3 system: mixed precision plus the learned
    preconditioner reaches |E - E_ref| < 1e-6 Ha in less wall time than the
    plain FP64 Teter-preconditioned minimiser on the same GPU."""
    import time
    from paper_1708_03621_gb300 import jdft, learned
    m = jdft.Mlp(learned.load_weights())
    o, g = _small()
    C0 = torch.tensor(o.coeffs(16), device="cuda")
    t = {}
    for label, pr, pc in (("fp64+teter", "fp64", "teter"), ("bf16x3+mlp", "bf16x3", "mlp")):
        best = None
        for _ in range(2):   # the first run includes one-time set-up
            C = C0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = jdft.jdft_minimize_bands(g.basis, 0, C, tol=1e-6, max_iter=3000, precond=pc, prec=pr,
                                           mlp=m if pc == "mlp" else None)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
            assert abs(rep["energy"] - GOLDEN["E_ref"]) < 1e-6
        t[label] = best
    assert t["bf16x3+mlp"] < t["fp64+teter"], t


def test_network_ties_teter_on_a_heldout_cell():
    """Held-out cell of seed 2009 (L = 17.7 bohr, 88 bands, 23 703 plane waves,
    80^3 box; the committed weights were trained on seeds 1000-1029): with the
    same BF16x3 schedule the network and Teter's preconditioner need about as
    many iterations (measured 163 and 160) and reach the same energy; the
    network does not beat Teter in iterations.  Mixed precision with either
    is faster than plain FP64 with Teter."""
    import time
    from paper_1708_03621_gb300 import jdft, learned
    from synth import training_cells
    w = [c for c in training_cells(10, 2000) if c.name == "train2009"][0]
    m = jdft.Mlp(learned.load_weights())
    b = learned.build_cell(w, "cuda")
    C0 = torch.tensor(learned.start_block(b, w), device="cuda")
    res = {}
    for label, pr, pc in (("bf16x3+teter", "bf16x3", "teter"), ("bf16x3+mlp", "bf16x3", "mlp"),
                          ("fp64+teter", "fp64", "teter")):
        C = C0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = jdft.jdft_minimize_bands(b, 0, C, tol=1e-6, max_iter=3000, precond=pc, prec=pr,
                                       mlp=m if pc == "mlp" else None)
        res[label] = (time.perf_counter() - t0, rep)
        assert rep["converged"], (label, rep)
    E = {k: v[1]["energy"] for k, v in res.items()}
    assert abs(E["bf16x3+mlp"] - E["fp64+teter"]) < 1e-6 and abs(E["bf16x3+teter"] - E["fp64+teter"]) < 1e-6
    its = {k: v[1]["iterations"] for k, v in res.items()}
    assert res["bf16x3+mlp"][1]["precond_fallback"] == 0
    assert 0.75 * its["bf16x3+teter"] < its["bf16x3+mlp"] < 1.25 * its["bf16x3+teter"], its
    assert res["bf16x3+mlp"][0] < res["fp64+teter"][0] and res["bf16x3+teter"][0] < res["fp64+teter"][0], res
    b.close()
