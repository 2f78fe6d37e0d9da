"""GPU parity of the Boltzmann log-partition (forward) and its gradient (backward)."""
import numpy as np
import pytest

import oracle
from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402

BETAS = list(inputs.LOGZ_BETAS)
RTOL = 1e-6


def run_forward(Qb, betas):
    Qd = torch.from_numpy(np.ascontiguousarray(Qb)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    return qb.qbf_logz(Qd.data_ptr(), Qb.shape[1], qb.dtype_code(Qd), Qb.shape[0], betas, s)


def run_backward(Qb, betas, upstream=None):
    Qd = torch.from_numpy(np.ascontiguousarray(Qb)).cuda()
    batch, n = Qb.shape[0], Qb.shape[1]
    grad = torch.empty((batch, n, n), dtype=torch.float64, device="cuda")
    mom = torch.empty((batch, len(betas), n, n), dtype=torch.float64, device="cuda")
    up = None if upstream is None else torch.tensor(upstream, dtype=torch.float64).cuda()
    s = torch.cuda.current_stream().cuda_stream
    qb.qbf_logz_backward(Qd.data_ptr(), n, qb.dtype_code(Qd), batch, betas,
                         None if up is None else up.data_ptr(), grad.data_ptr(), mom.data_ptr(), s)
    torch.cuda.synchronize()
    return grad.cpu().numpy(), mom.cpu().numpy()


@pytest.mark.parametrize("n", [2, 3, 5, 8, 11, 14, 17])
def test_logz_forward_and_moments_against_oracle(n):
    rng = np.random.default_rng(900 + n)
    Qb = np.triu(rng.normal(0, 1 / np.sqrt(n), size=(3, n, n))).astype(np.float32)
    lz, vmin, am = run_forward(Qb, BETAS)
    grad, mom = run_backward(Qb, BETAS)
    for b in range(3):
        olz, oE, ov, oa = oracle.logz(Qb[b], BETAS)
        assert (vmin[b], am[b]) == (ov, oa)
        for j, beta in enumerate(BETAS):
            assert abs(lz[b][j] - olz[j]) <= RTOL * abs(olz[j]) + 1e-9, (b, beta)
            assert np.max(np.abs(mom[b, j] - oE[j]) - RTOL * np.abs(oE[j])) <= 1e-9, (b, beta)
        want = sum(-beta * oE[j] for j, beta in enumerate(BETAS))
        assert np.allclose(grad[b], want, rtol=RTOL, atol=1e-9)


@pytest.mark.parametrize("betas", [[0.2, 1.0, 3.0, 7.0], [0.05, 0.1, 0.3, 1.0, 2.0, 5.0, 10.0]])
def test_logz_many_betas_against_oracle(betas):
    """More betas than one moment walk takes (three): the backward splits
    them over several launches (3 + 1, 3 + 3 + 1), the forward predicates
    the Z walk compiled for eight."""
    n = 11
    rng = np.random.default_rng(950 + len(betas))
    Qb = np.triu(rng.normal(0, 1 / np.sqrt(n), size=(2, n, n))).astype(np.float32)
    lz, vmin, am = run_forward(Qb, betas)
    grad, mom = run_backward(Qb, betas)
    for b in range(2):
        olz, oE, ov, oa = oracle.logz(Qb[b], betas)
        assert (vmin[b], am[b]) == (ov, oa)
        for j, beta in enumerate(betas):
            assert abs(lz[b][j] - olz[j]) <= RTOL * abs(olz[j]) + 1e-9, (b, beta)
            assert np.max(np.abs(mom[b, j] - oE[j]) - RTOL * np.abs(oE[j])) <= 1e-9, (b, beta)
        want = sum(-beta * oE[j] for j, beta in enumerate(betas))
        assert np.allclose(grad[b], want, rtol=RTOL, atol=1e-9)


def test_logz_integer_and_f64_inputs():
    rng = np.random.default_rng(4)
    for Qb in (rng.integers(-3, 4, size=(2, 10, 10)).astype(np.int32),
               np.triu(rng.uniform(-1, 1, size=(2, 9, 9)))):
        lz, vmin, am = run_forward(Qb, [0.5, 2.0])
        _, mom = run_backward(Qb, [0.5, 2.0])
        for b in range(2):
            olz, oE, ov, oa = oracle.logz(Qb[b], [0.5, 2.0])
            assert np.allclose(lz[b], olz, rtol=RTOL, atol=1e-9)
            assert np.allclose(mom[b], oE, rtol=RTOL, atol=1e-9)


def test_logz_upstream_weights_gradient():
    n = 9
    Qb = inputs.config_logz(count=2, n=n, seed=5)
    up = [[0.3, -1.0, 2.0], [1.5, 0.0, -0.25]]
    grad, mom = run_backward(Qb, BETAS, upstream=up)
    for b in range(2):
        want = sum(up[b][j] * (-beta) * mom[b, j] for j, beta in enumerate(BETAS))
        assert np.allclose(grad[b], want, rtol=1e-12, atol=1e-15)


def test_logz_diagonal_closed_form():
    d = np.array([0.7, -0.2, 0.0, -1.3, 0.4, 0.9], dtype=np.float64)
    Qb = np.diag(d)[None]
    lz, _, _ = run_forward(Qb, BETAS)
    _, mom = run_backward(Qb, BETAS)
    for j, beta in enumerate(BETAS):
        assert abs(lz[0][j] - np.sum(np.log1p(np.exp(-beta * d)))) <= RTOL * abs(lz[0][j]) + 1e-9
        p = 1 / (1 + np.exp(beta * d))
        want = np.outer(p, p)
        want[np.diag_indices(6)] = p
        assert np.allclose(mom[0, j], want, rtol=RTOL, atol=1e-9)


def test_autograd_wrappers():
    Qb = torch.from_numpy(inputs.config_logz(count=2, n=10, seed=8)).cuda().requires_grad_(True)
    out = qb.logz(Qb, BETAS)
    w = torch.tensor([[1.0, 0.5, 0.1], [0.0, 2.0, 1.0]], dtype=torch.float64, device="cuda")
    (out * w).sum().backward()
    g = Qb.grad.detach().cpu().numpy()
    grad, _ = run_backward(Qb.detach().cpu().numpy(), BETAS, upstream=w.cpu().numpy().tolist())
    assert np.allclose(g, grad.astype(np.float32), rtol=1e-6, atol=1e-7)
    Q2 = torch.from_numpy(inputs.config_logz(count=3, n=12, seed=9)).cuda().requires_grad_(True)
    m = qb.qubo_min(Q2)
    m.sum().backward()
    for b in range(3):
        v, a = oracle.brute_min(Q2[b].detach().cpu().numpy())
        assert m[b].item() == v
        x = np.array([(a >> i) & 1 for i in range(12)], dtype=np.float32)
        assert np.array_equal(Q2.grad[b].cpu().numpy(), np.outer(x, x))


def test_logz_config_64x28():
    """64 instances at n = 28, N(0, 1/n): forward for all, oracle on a sample, FD on entries."""
    Qb = inputs.config_logz()
    lz, vmin, am = run_forward(Qb, BETAS)
    lz = np.array(lz)
    n = 28
    for b in range(64):
        # properties at any size: the minimum state bounds log Z from below, the
        # count of states from above; log Z decreases in beta past the minimum
        for j, beta in enumerate(BETAS):
            assert -beta * vmin[b] <= lz[b, j] <= -beta * vmin[b] + n * np.log(2) + 1e-9
        assert vmin[b] == oracle.evaluate(Qb[b], am[b])
    # one instance in full against the FP64 oracle
    olz, oE, ov, oa = oracle.logz(Qb[0], BETAS)
    assert np.allclose(lz[0], olz, rtol=RTOL, atol=1e-9)
    grad, mom = run_backward(Qb[:1], BETAS)
    for j in range(3):
        assert np.allclose(mom[0, j], oE[j], rtol=RTOL, atol=1e-9), j
    # central differences of the GPU forward (h = 1e-3) against the GPU backward
    h = 1e-3
    for (i, k) in [(0, 0), (3, 17), (27, 27), (10, 20)]:
        Qp, Qm = Qb[:1].copy(), Qb[:1].copy()
        Qp[0, i, k] += h
        Qm[0, i, k] -= h
        fp = np.array(run_forward(Qp, BETAS)[0][0])
        fm = np.array(run_forward(Qm, BETAS)[0][0])
        # Qp/Qm are FP32: use the perturbation actually stored
        hh = (np.float64(Qp[0, i, k]) - np.float64(Qm[0, i, k])) / 2
        fd = (fp - fm) / (2 * hh)
        an = np.array([-beta * mom[0, j, i, k] for j, beta in enumerate(BETAS)])
        assert np.all(np.abs(fd - an) <= 1e-3 * np.maximum(np.abs(an), 1e-2)), (i, k, fd, an)


def test_logz_config_64x28_four_instances_against_stored_oracle():
    """Four of the 64 n = 28 instances (0, 21, 42, 63) in full against the
    stored FP64 oracle: log Z and E[x x^T] at beta in {0.1, 1, 10} to 1e-6
    relative, and the gradient -beta E[x_i x_j] against central differences
    of the oracle's log Z (h = 1e-3) to 1e-4 relative."""
    import json
    import os

    from conftest import GOLDEN

    g = json.load(open(os.path.join(GOLDEN, "config_logz_n28.json")))
    assert g["betas"] == BETAS
    Qall = inputs.config_logz()
    idx = [e["index"] for e in g["instances"]]
    Qb = Qall[idx]
    lz, vmin, am = run_forward(Qb, BETAS)
    grad, mom = run_backward(Qb, BETAS)
    for k, e in enumerate(g["instances"]):
        assert (vmin[k], am[k]) == (e["min"], e["argmin"])
        for j, beta in enumerate(BETAS):
            assert abs(lz[k][j] - e["logz"][j]) <= RTOL * abs(e["logz"][j]) + 1e-9, (k, beta)
            oE = np.array(e["moment"][j])
            assert np.allclose(mom[k, j], oE, rtol=RTOL, atol=1e-9), (k, beta)
        want = sum(-beta * np.array(e["moment"][j]) for j, beta in enumerate(BETAS))
        assert np.allclose(grad[k], want, rtol=RTOL, atol=1e-9)
    cd = g["central_differences"]
    k0 = idx.index(cd["instance"])
    for ent in cd["entries"]:
        i, j2 = ent["i"], ent["j"]
        for jb, beta in enumerate(BETAS):
            an = -beta * mom[k0, jb, i, j2]
            fd = ent["dlogz"][jb]
            assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-2), (i, j2, beta, fd, an)
