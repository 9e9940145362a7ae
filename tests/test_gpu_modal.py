"""GPU parity of the modal raw projections <<B_l|Q_pqr>> (Sec. 3.5) against
the FP64 oracle's x-space sums (pinned by a Fourier-space brute force and by
the reduction to the standard estimator), for the CUDA-core FP32 path and the
split-FP16 tensor-core path.  Gate: |dS| / max(|S|, rms_l) <= 1e-5."""
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


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
@pytest.mark.parametrize("ells", [(0, 2, 4), (0, 4)])
def test_modal_matches_oracle(torch_cuda, ora, prec, ells):
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    n, nmodes = 32, 6
    kf = 2 * np.pi / BOX
    dk, amp = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 31)
    R = bsp.bsp_modal_radial_powerlaw(n, BOX, nmodes, kf, 14 * kf, amp, -1.5, True)
    est = bsp.Modal(n, BOX, R, ells, prec=prec)
    S = est.compute(torch.from_numpy(dk).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    if prec != "fp32":
        assert bsp.bsp_device_status(est.plan) == 0
    est.close()
    full = ora.full_from_half(dk.astype(np.complex128), n)
    slots = sorted(set(ells) | ({2} if 4 in ells else set()) | {0})
    M = ora.modal_fields(full, n, R, slots)
    trip = ora.modal_triplets(nmodes)
    So = ora.modal_raw(M, ells, trip) / (n ** 3 * BOX ** 9)
    rms = np.sqrt(np.mean(So ** 2, axis=1, keepdims=True))
    err = np.max(np.abs(S - So) / np.maximum(np.abs(So), rms))
    print("modal %s ells=%s gate %.3g" % (prec, ells, err))
    assert err <= 1e-5
