"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Gate (FP32 contraction): for every bin and multipole,
    |B_gpu - B_ora| / max(|B_ora|, rms_l) <= 1e-5,
rms_l the root mean square of B_ora over the bins of that multipole.
Counts and the bin list are integers and must match exactly.
"""
import math

import numpy as np
import pytest

from paper_1708_05303_gb300.synth import FieldModel, delta_k_from_real, linear_edges, make_field

pytestmark = pytest.mark.gpu
BOX = 1000.0
TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_05303_gb300 import build

    build.build()
    return torch


def gate(B_gpu, B_ora):
    rms = np.sqrt(np.mean(B_ora ** 2, axis=1, keepdims=True))
    den = np.maximum(np.abs(B_ora), rms)
    return np.max(np.abs(B_gpu - B_ora) / den)


def run_gpu(torch, dk, n, edges, ells, prec="fp32"):
    from paper_1708_05303_gb300.bsp import Bispectrum

    est = Bispectrum(n, BOX, edges, ells, prec=prec)
    d = torch.from_numpy(np.ascontiguousarray(dk.astype(np.complex64))).cuda()
    B = est.compute(d).cpu().numpy()
    T = est.raw().cpu().numpy()
    torch.cuda.synchronize()
    out = dict(bins=est.bins, counts=est.counts, B=B, T=T)
    est.close()
    return out


CASES = [
    # (n, edges, ells, seed) -- pruned and unpruned geometries, mixed radices
    (16, [1, 3, 5, 7], (0, 2, 4), 1),
    (16, [1, 4, 7, 10, 13], (0, 2, 4), 2),      # edges beyond n/2: no pruning, Nyquist planes, wrap-around
    (24, [1, 3, 5, 7, 9, 11], (0, 2), 3),       # 2^3 * 3
    (40, [2, 5, 8, 11, 14], (0, 4), 4),         # 2^3 * 5
    (32, linear_edges(8), (0, 2, 4), 5),
    (48, linear_edges(10), (0, 2, 4), 6),
]


@pytest.mark.parametrize("n,edges,ells,seed", CASES)
def test_fp32_matches_oracle(torch_cuda, ora, n, edges, ells, seed):
    model = FieldModel(n=n, box=BOX, sigma_g=0.3)
    dk, _ = make_field(model, seed)
    g = run_gpu(torch_cuda, dk, n, edges, ells)
    r = ora.bispectrum(dk.astype(np.complex128), n, BOX, edges, ells)
    assert np.array_equal(g["bins"], r["bins"])
    assert np.array_equal(g["counts"], r["counts"])
    err = gate(g["B"], r["B"])
    assert err <= TOL, err
    # raw sums against the oracle's, on the round-off scale of the summand
    scale = np.sqrt(r["sumsq"])
    assert np.max(np.abs(g["T"] - r["T"]) / np.maximum(np.abs(r["T"]), scale)) < 1e-5


def test_config_64_16_shells(torch_cuda, ora):
    """The 64^3 / 16-shell workload: every bin and l."""
    n = 64
    edges = linear_edges(16)
    model = FieldModel(n=n, box=BOX)
    dk, _ = make_field(model, 1709)
    g = run_gpu(torch_cuda, dk, n, edges, (0, 2, 4))
    r = ora.bispectrum(dk.astype(np.complex128), n, BOX, edges)
    assert len(r["bins"]) == 564
    assert np.array_equal(g["bins"], r["bins"])
    assert np.array_equal(g["counts"], r["counts"])
    assert gate(g["B"], r["B"]) <= TOL


def test_worked_example_on_gpu(torch_cuda):
    """delta = sum of three cosines: only bin (2,1,0) is nonzero and equals
    2 (V/2)^3 w_l(mu_3) / (V N_abc) (Eq. Bisp_ell_restrict)."""
    n = 16
    V = BOX ** 3
    q1, q2 = (2, 0, 1), (0, 3, 1)
    q3 = tuple(-(u + v) for u, v in zip(q1, q2))
    x = np.indices((n, n, n)).reshape(3, -1).T
    d = sum(np.cos(2 * np.pi * (x @ np.array(q)) / n) for q in (q1, q2, q3)).reshape(n, n, n)
    dk = delta_k_from_real(d, BOX)
    g = run_gpu(torch_cuda, dk, n, [1, 2.5, 4, 5.5], (0, 2, 4))
    mu2 = 4.0 / 17.0
    w = {0: 1.0, 2: 2.5 * (3 * mu2 - 1), 4: 1.125 * (35 * mu2 ** 2 - 30 * mu2 + 3)}
    bins = [tuple(b) for b in g["bins"]]
    bi = bins.index((2, 1, 0))
    for li, ell in enumerate((0, 2, 4)):
        want = 2 * (V / 2) ** 3 * w[ell] / (V * g["counts"][bi])
        assert abs(g["B"][li, bi] - want) <= 1e-5 * abs(2 * (V / 2) ** 3 / (V * g["counts"][bi]))
        others = np.delete(g["B"][li], bi)
        assert np.max(np.abs(others)) <= 1e-5 * abs(want) + 1e-6 * (V / 2) ** 2


def test_host_path_equals_device_path(torch_cuda):
    from paper_1708_05303_gb300.bsp import Bispectrum

    torch = torch_cuda
    n = 32
    edges = linear_edges(6)
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 77)
    est = Bispectrum(n, BOX, edges, (0, 2, 4), host_staging=True)
    B_dev = est.compute(torch.from_numpy(dk).cuda()).cpu().numpy()
    host = torch.from_numpy(np.ascontiguousarray(dk)).pin_memory()
    out = torch.empty(B_dev.shape, dtype=torch.float64).pin_memory()
    est.compute_host(host.numpy(), out.numpy())
    assert np.array_equal(out.numpy(), B_dev)
    est.close()


def test_repeat_is_deterministic(torch_cuda):
    from paper_1708_05303_gb300.bsp import Bispectrum

    torch = torch_cuda
    n = 32
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 8)
    est = Bispectrum(n, BOX, linear_edges(8), (0, 2, 4))
    d = torch.from_numpy(dk).cuda()
    a = est.compute(d).clone()
    b = est.compute(d).clone()
    assert torch.equal(a, b)
    est.close()
