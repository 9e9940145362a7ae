"""GPU skew-spectrum multipoles (Sec. 3.3, convolution form) against the FP64
oracle on the same complex64 spectrum.  The GPU path is an FP32 inverse FFT,
an FP32 square and forward FFT, and FP32 cross products summed in FP64; the
gate is 1e-5 of max(|S|, rms over shells), on pruned and unpruned shell
sets, with bit-identical repeats."""
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


@pytest.mark.parametrize("n,nsh,width", [(64, 16, 2.0), (48, 12, 2.0), (128, 20, 2.0)])
def test_skew_matches_oracle(torch_cuda, ora, n, nsh, width):
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    edges = linear_edges(nsh, width)
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 1708 + 3 * n)
    est = bsp.Bispectrum(n, BOX, edges, (0, 2, 4))
    d = torch.from_numpy(dk).cuda()
    S, Nk = est.skew(d)
    S1 = S.cpu().numpy().copy()
    S2, _ = est.skew(d)
    est.close()
    r = ora.skew_spectrum(dk.astype(np.complex128), n, BOX, edges)
    assert np.array_equal(Nk.cpu().numpy(), r["Nk"])
    rms = np.sqrt(np.mean(r["S"] ** 2, axis=1, keepdims=True))
    e = float(np.max(np.abs(S1 - r["S"]) / np.maximum(np.abs(r["S"]), rms)))
    print("skew %d^3, %d shells: gate %.3g" % (n, nsh, e))
    assert e <= 1e-5
    assert np.array_equal(S1, S2.cpu().numpy())
