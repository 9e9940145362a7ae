"""BSP_FULL_TENSOR: T^l[a; b >= c] for every assignment of the Legendre leg
(Sec. 3.1 weights the largest side; the full tensor lets a first-index
convention be read off as well), against the FP64 oracle on the same bins,
gated at 1e-5 of max(|B|, rms_l), on the FP32 and split-FP16 paths; the
entries with a as the largest side equal the standard plan's."""
import numpy as np
import pytest

from paper_1708_05303_gb300.synth import FieldModel, linear_edges, make_field

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


def gate(B_gpu, B_ora):
    rms = np.sqrt(np.mean(B_ora ** 2, axis=1, keepdims=True))
    return np.max(np.abs(B_gpu - B_ora) / np.maximum(np.abs(B_ora), rms))


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
def test_full_tensor_matches_oracle(torch_cuda, ora, prec):
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    n, edges, ells = 32, linear_edges(8), (0, 2, 4)
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 1712)
    d = torch.from_numpy(dk).cuda()
    std = bsp.Bispectrum(n, BOX, edges, ells, prec=prec)
    B_std = std.compute(d).cpu().numpy()
    full = bsp.Bispectrum(n, BOX, edges, ells, prec=prec, full_tensor=True, counts_from=std)
    B = full.compute(d).cpu().numpy()
    torch.cuda.synchronize()
    assert bsp.bsp_device_status(full.plan) == 0
    bins = [tuple(int(v) for v in t) for t in full.bins]
    std_bins = [tuple(int(v) for v in t) for t in std.bins]
    # every assignment of the Legendre leg of every valid bin, and nothing else
    want = sorted({(t[k], max(t[(k + 1) % 3], t[(k + 2) % 3]), min(t[(k + 1) % 3], t[(k + 2) % 3]))
                   for t in std_bins for k in range(3)})
    assert bins == want and any(a < b for (a, b, c) in bins)
    r = ora.bispectrum(dk.astype(np.complex128), n, BOX, edges, ells, bins=bins)
    assert np.array_equal(full.counts, r["counts"])
    err = gate(B, r["B"])
    print("full tensor %s: %d bins, gate error %.3g" % (prec, len(bins), err))
    assert err <= 1e-5
    # the largest-side entries are the standard plan's outputs (same arithmetic per bin)
    idx = [bins.index(t) for t in std_bins]
    assert gate(B[:, idx], B_std) <= 1e-5
    full.close()
    std.close()
