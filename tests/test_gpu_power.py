"""GPU power-spectrum multipoles (Sec. 2, Eq. PowSpecMultipole) against the
FP64 oracle on the same complex64 spectrum: the GPU forms each mode's
w_l |delta|^2 in FP32 (relative rounding ~1e-7) and sums in FP64, so the gate
is 1e-6 of max(|P|, rms over shells); mode counts exactly; pruned and unpruned
geometries; shot noise; bit-identical repeats."""
import numpy as np
import pytest

from paper_1708_05303_gb300.synth import FieldModel, linear_edges, make_field
from particle_input import particle_delta

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


def gate(P, ref):
    rms = np.sqrt(np.mean(ref ** 2, axis=1, keepdims=True))
    return float(np.max(np.abs(P - ref) / np.maximum(np.abs(ref), rms)))


@pytest.mark.parametrize("n,nsh,width", [(64, 16, 2.0), (32, 13, 2.0), (48, 10, 1.5)])
def test_power_matches_oracle(torch_cuda, ora, n, nsh, width):
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    edges = linear_edges(nsh, width)
    dk, _ = make_field(FieldModel(n=n, box=BOX), 1708 + n)
    est = bsp.Bispectrum(n, BOX, edges, (0, 2, 4))
    d = torch.from_numpy(dk).cuda()
    P, Nk = est.power(d)
    P1 = P.cpu().numpy().copy()
    P2, _ = est.power(d)
    est.close()
    r = ora.power_multipoles(dk.astype(np.complex128), n, BOX, edges)
    assert np.array_equal(Nk.cpu().numpy(), r["Nk"])
    e = gate(P1, r["P"])
    print("power %d^3, %d shells: gate %.3g" % (n, nsh, e))
    assert e <= 1e-6
    assert np.array_equal(P1, P2.cpu().numpy())   # deterministic


def test_power_shot_noise_256(torch_cuda, ora):
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    n = 256
    edges = linear_edges(32)
    dk, npart, nbar = particle_delta(FieldModel(n=n, box=BOX, sigma_g=0.3), 1708 + 1)
    est = bsp.Bispectrum(n, BOX, edges, (0, 2, 4), shot_noise=True)
    P, Nk = est.power(torch.from_numpy(dk).cuda(), nbar=nbar)
    P = P.cpu().numpy()
    est.close()
    r = ora.power_multipoles(dk.astype(np.complex128), n, BOX, edges, nbar=nbar)
    assert np.array_equal(Nk.cpu().numpy(), r["Nk"])
    e = gate(P, r["P"])
    print("power 256^3 with shot noise: gate %.3g, shot/P0 at the last shell %.3g"
          % (e, r["shot"][0, -1] / r["P_raw"][0, -1]))
    assert e <= 1e-6
    assert np.max(np.abs(r["shot"][0] - 1.0 / nbar)) <= 1e-12 / nbar
