"""GPU preconditioner network against the FP64 oracle network (BF16 weights on
both sides, so only the FP32 activations differ), the training rows against
the oracle's residual/correction blocks, and the trained-versus-untrained
behaviour of the band minimiser."""
import numpy as np
import pytest

from oracle import minimize as mn
from oracle import mlp as omlp
from oracle import planewave as pw
from synth import mlp_init
from tests.systems import GpuSystem, OracleSystem, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

rng = np.random.default_rng(21)


def bf16_round(x):
    """Round float values to the nearest bfloat16 (ties to even), as FP64 values."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def rows_np(n):
    X = np.column_stack([rng.uniform(0, 20, n), rng.uniform(0, 2, n), rng.uniform(0, 3, n)])
    return np.column_stack([X, rng.uniform(0.1, 2.0, n), rng.normal(0, 1, n)]).astype(np.float32)


def test_forward_matches_oracle_with_bf16_weights():
    from paper_1708_03621_gb300 import jdft
    theta = mlp_init(11).astype(np.float32)
    m = jdft.Mlp(theta)
    R = rows_np(5000)
    K = torch.empty(5000, dtype=torch.float32, device="cuda")
    jdft.jdft_mlp_forward(m, torch.tensor(R[:, :3], device="cuda"), K)
    ref, _ = omlp.forward(bf16_round(theta), R[:, :3].astype(np.float64))
    assert np.max(np.abs(K.cpu().numpy() - ref) / ref) < 2e-5


def test_loss_and_gradient_match_oracle():
    from paper_1708_03621_gb300 import jdft
    theta = mlp_init(12).astype(np.float32)
    theta[-1] = 0.2
    m = jdft.Mlp(theta)
    R = rows_np(3000)   # several tiles and blocks, ragged last tile
    g = torch.empty(jdft.MLP_NPARAM, dtype=torch.float32, device="cuda")
    L = torch.empty(2, dtype=torch.float64, device="cuda")
    jdft.jdft_mlp_loss_grad(m, torch.tensor(R, device="cuda"), g, L)
    tb = bf16_round(theta)
    Rd = R.astype(np.float64)
    assert abs(L[0].item() - omlp.loss(tb, Rd)) < 1e-5 * max(1.0, abs(omlp.loss(tb, Rd)))
    ref = omlp.grad(tb, Rd)
    got = g.cpu().numpy().astype(np.float64)
    cos = got @ ref / np.linalg.norm(got) / np.linalg.norm(ref)
    assert cos > 0.99999
    assert np.linalg.norm(got - ref) < 1e-4 * np.linalg.norm(ref)


def test_adam_training_reduces_loss():
    from paper_1708_03621_gb300 import jdft, learned
    m = jdft.Mlp(mlp_init(13))
    R = rows_np(20000)
    R[:, 4] = R[:, 3] * (1.0 / (1.0 + 0.5 * R[:, 0]))    # target K = 1/(1 + x/2)
    rows = torch.tensor(R, device="cuda")
    before = learned.evaluation_loss(m, rows)
    hist = learned.train(m, rows, epochs=15, batch=4096, lr=3e-3, log=lambda *_: None)
    after = learned.evaluation_loss(m, rows)
    # the loss floor is -sum(q^2/a)/sum(a): reach most of the way there
    floor = float(-(R[:, 4].astype(np.float64) ** 2 / R[:, 3]).sum() / R[:, 3].sum())
    assert after < before and (after - floor) < 0.05 * (before - floor)
    assert hist[-1] < hist[0]


def test_training_rows_match_oracle():
    from paper_1708_03621_gb300 import jdft
    w = workload("tiny_cubic")
    o = OracleSystem(w)
    g = GpuSystem(w, o.atoms)
    nb = 4
    Cst = mn.minimize_bands(o.basis, lambda X: pw.apply_H(o.basis, o.V, X, o.P, o.D), o.coeffs(nb).T,
                            tol=1e-10).C
    C = pw.lowdin(o.coeffs(nb, seed=5).T, o.basis.Omega)
    rows = jdft.jdft_mlp_rows(g.basis, 0, torch.tensor(np.ascontiguousarray(C.T), device="cuda"),
                              torch.tensor(np.ascontiguousarray(Cst.T), device="cuda"), stride=3, offset=1)
    got = rows.cpu().numpy().astype(np.float64)
    # oracle rows
    r, eps, Hs, G = mn.residual_norms(o.basis, C, pw.apply_H(o.basis, o.V, C, o.P, o.D))
    t = C - Cst @ (o.basis.Omega * (Cst.conj().T @ C))
    F = omlp.features(o.basis.T, mn.band_kinetic(o.basis, C), np.real(np.diag(Hs)))   # (npw, nb, 3)
    idx = np.arange(1, nb * o.basis.npw, 3)
    b, gg = idx // o.basis.npw, idx % o.basis.npw
    ref = np.column_stack([F[gg, b, 0], F[gg, b, 1], F[gg, b, 2], np.abs(G[gg, b]) ** 2,
                           (np.conj(G[gg, b]) * t[gg, b]).real])
    ref[:, 4] *= ref[:, 3].sum() / ref[:, 4].sum()     # the library's per-snapshot scaling
    assert got.shape == ref.shape
    scale = np.max(np.abs(ref), axis=0)
    assert np.max(np.abs(got - ref) / scale) < 1e-5


def test_network_preconditioner_converges_and_beats_unpreconditioned():
    """Minimiser with a network trained on the GPU (a few small cells) reaches
    the same energy as Teter and needs fewer iterations than no preconditioner."""
    from paper_1708_03621_gb300 import jdft, learned
    from synth import training_cells
    cells = training_cells(3, 3000, L_range=(8.0, 10.0), ecut=12.0)
    rows = learned.generate_rows(cells, rows_per_snapshot=20000, log=lambda *_: None)
    m = jdft.Mlp(mlp_init(7))
    learned.train(m, rows, epochs=12, batch=8192, lr=3e-3, log=lambda *_: None)
    w = workload("mid")
    o = OracleSystem(w)
    gsys = GpuSystem(w, o.atoms)
    its, Es = {}, {}
    for pc in ("teter", "mlp", "identity"):
        C = torch.tensor(o.coeffs(16), device="cuda")
        rep = jdft.jdft_minimize_bands(gsys.basis, 0, C, tol=1e-8, max_iter=3000, precond=pc,
                                       mlp=m if pc == "mlp" else None)
        assert rep["converged"], (pc, rep)
        its[pc], Es[pc] = rep["iterations"], rep["energy"]
    assert abs(Es["mlp"] - Es["teter"]) < 1e-6 and abs(Es["identity"] - Es["teter"]) < 1e-6
    assert its["mlp"] < its["identity"], its
    assert its["mlp"] < 1.5 * its["teter"], its


def test_committed_weights_on_the_48_cubed_system():
    """The committed network (trained on the GPU, cells L = 16-24 bohr) on the
    48^3 system it never saw: same energy as Teter within 1e-6 Ha, and fewer
    iterations than the unpreconditioned minimiser."""
    import json
    import os
    from paper_1708_03621_gb300 import jdft, learned
    wts = learned.load_weights()
    assert wts is not None and wts.shape == (jdft.MLP_NPARAM,)
    m = jdft.Mlp(wts)
    w = workload("small")
    o = OracleSystem(w)
    g = GpuSystem(w, o.atoms)
    golden = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                         "small_eigs.json")))
    its = {}
    for pc in ("mlp", "identity"):
        C = torch.tensor(o.coeffs(16), device="cuda")
        rep = jdft.jdft_minimize_bands(g.basis, 0, C, tol=1e-8, max_iter=3000, precond=pc, prec="tf32x3",
                                       mlp=m if pc == "mlp" else None)
        assert rep["converged"], (pc, rep)
        assert abs(rep["energy"] - golden["E_ref"]) < 1e-6
        its[pc] = rep["iterations"]
    assert its["mlp"] < its["identity"], its
