"""GPU batch runner (uneven grids, CUDA graphs, autotuner) and FP64
covariance, against the FP64 oracle.

Every row must match the oracle's multipoles for that mock (FP32 gate 1e-5),
the covariance must match the oracle's two-pass covariance of the oracle's
rows, and the graphs must give the same rows as plain bsp_compute calls.
"""
import numpy as np
import pytest

from paper_1708_05303_gb300.synth import FieldModel, make_field

pytestmark = pytest.mark.gpu
BOX = 1000.0


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_05303_gb300 import build

    build.build()
    return torch


def mocks(sizes, count):
    out = []
    for m in range(count):
        rng = np.random.Generator(np.random.PCG64(1708 * 1000 + m + 104729))
        ns, f = float(rng.uniform(-2.0, -1.0)), float(rng.uniform(0.5, 0.9))
        n = sizes[m % len(sizes)]
        dk, _ = make_field(FieldModel(n=n, box=BOX, amp=2.0e4, n_s=ns, f=f, sigma_g=0.3), 1708 * 1000 + m)
        out.append((m % len(sizes), dk))
    return out


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
def test_batch_rows_and_covariance(torch_cuda, ora, prec):
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    sizes = (24, 32, 40)
    edges = [1, 2, 3, 4, 5, 6, 7]          # width k_f: alias-free and the same bins on all three grids
    ms = mocks(sizes, 9)
    batch = bsp.Batch(sizes, BOX, edges, (0, 2, 4), prec=prec, autotune=True)
    hosts = [torch.from_numpy(dk).pin_memory() for _, dk in ms]
    rows = batch.run(hosts, [s for s, _ in ms])
    mean, cov = batch.covariance(rows)
    torch.cuda.synchronize()
    rows_h = rows.cpu().numpy()
    tol = 1e-5
    ora_rows = []
    for (si, dk), row in zip(ms, rows_h):
        r = ora.bispectrum(dk.astype(np.complex128), sizes[si], BOX, edges)
        assert np.array_equal(r["bins"], batch.bins)
        B = row.reshape(3, -1)
        rms = np.sqrt(np.mean(r["B"] ** 2, axis=1, keepdims=True))
        assert np.max(np.abs(B - r["B"]) / np.maximum(np.abs(r["B"]), rms)) <= tol
        ora_rows.append(r["B"].ravel())
    ora_rows = np.array(ora_rows)
    C_ora = ora.covariance(ora_rows)
    scale = np.sqrt(np.outer(np.diag(C_ora), np.diag(C_ora)))
    assert np.max(np.abs(cov.cpu().numpy() - C_ora) / scale) <= 50 * tol
    # the covariance kernel itself against numpy on the same rows
    assert np.allclose(cov.cpu().numpy(), np.cov(rows_h, rowvar=False), rtol=1e-9, atol=1e-12 * np.abs(C_ora).max())
    assert np.allclose(mean.cpu().numpy(), rows_h.mean(axis=0), rtol=1e-12, atol=0)
    print(prec, "tuning", batch.tuning)
    batch.close()


def test_graph_replay_equals_direct_compute(torch_cuda):
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    sizes = (32, 40)
    edges = [1, 3, 5, 7, 9]
    ms = mocks(sizes, 4)
    batch = bsp.Batch(sizes, BOX, edges, (0, 2, 4), autotune=False)
    rows = batch.run([torch.from_numpy(dk).pin_memory() for _, dk in ms], [s for s, _ in ms]).cpu().numpy()
    batch.close()
    for (si, dk), row in zip(ms, rows):
        est = bsp.Bispectrum(sizes[si], BOX, edges, (0, 2, 4))
        B = est.compute(torch.from_numpy(dk).cuda()).cpu().numpy()
        est.close()
        assert np.allclose(row, B.ravel(), rtol=1e-12, atol=0)
