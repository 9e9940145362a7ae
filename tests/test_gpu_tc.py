"""GPU parity of the tensor-core (tcgen05) contraction against the FP64 oracle.

split_f16: power-of-two scaled FP16 hi + lo split of both operands (22
significant bits), three products, FP32 accumulation at the library's
default chunk of 64 points (the benchmarked settings): gated at 1e-5 of
max(|B|, rms_l) like the FP32 path on every field of the benchmark's model
(sigma_g = 0.3) and on the unscaled 64^3 field (sigma_g^2 ~ 82, below).
split_bf16: the BF16 hi + lo split (16 significant bits; its representation
error alone is ~5e-5 of the gate scale on small grids, computed exactly on
the CPU for the same inputs), gated at 2e-4 and reported.
bf16: one product; its error is reported and only bounded loosely.
Every run also checks the kernels' device error word.
"""
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


def run(torch, dk, n, edges, ells, prec, chunk=None):
    from paper_1708_05303_gb300 import bsp

    est = bsp.Bispectrum(n, BOX, edges, ells, prec=prec)
    if chunk:
        bsp.bsp_set_accumulation_chunk(est.plan, chunk)
    B = est.compute(torch.from_numpy(np.ascontiguousarray(dk)).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    status = bsp.bsp_device_status(est.plan)
    bins = est.bins.copy()
    est.close()
    return bins, B, status


CASES = [
    (16, [1, 3, 5, 7], (0, 2, 4), 1),
    (32, linear_edges(8), (0, 2, 4), 5),
    (24, [1, 3, 5, 7, 9, 11], (0, 2), 3),
    (64, linear_edges(16), (0, 2, 4), 1709),
    (48, linear_edges(10), (0, 2, 4), 6),
]

# split-BF16 keeps 16 significant bits: its representation error alone is
# ~5e-5 of the gate scale on these grids (computed exactly on the CPU for the
# same inputs), so it is reported and bounded, not gated at 1e-5.
GATES = {"split_f16": 1e-5, "split_bf16": 2e-4}


@pytest.mark.parametrize("prec", ["split_f16", "split_bf16"])
@pytest.mark.parametrize("n,edges,ells,seed", CASES)
def test_split_matches_oracle(torch_cuda, ora, n, edges, ells, seed, prec):
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), seed)
    bins, B, status = run(torch_cuda, dk, n, edges, ells, prec)
    assert status == 0
    r = ora.bispectrum(dk.astype(np.complex128), n, BOX, edges, ells)
    assert np.array_equal(bins, r["bins"])
    err = gate(B, r["B"])
    print("%s n=%d gate error %.3g" % (prec, n, err))
    assert err <= GATES[prec], err


def test_unscaled_field_64(torch_cuda, ora):
    """The 64^3 / 16-shell case on the unscaled field (sigma_g^2 ~ 82, far
    from Gaussian).  On this field the split-FP16 error is set by the tensor
    core's FP32 accumulation, which truncates every addend of an MMA below
    the largest one (a CPU emulation of the split arithmetic gives 1.2e-6
    with exact accumulation): drained every 256 points it departed by
    1.1e-5; at the library's 64-point default both paths meet 1e-5."""
    n, edges, ells = 64, linear_edges(16), (0, 2, 4)
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=None), 1709)
    r = ora.bispectrum(dk.astype(np.complex128), n, BOX, edges, ells)
    bins, B32, _ = run(torch_cuda, dk, n, edges, ells, "fp32")
    assert np.array_equal(bins, r["bins"])
    e32 = gate(B32, r["B"])
    _, Bs, status = run(torch_cuda, dk, n, edges, ells, "split_f16")
    assert status == 0
    es = gate(Bs, r["B"])
    print("unscaled 64^3: fp32 gate error %.3g, split_f16 %.3g" % (e32, es))
    assert e32 <= 1e-5
    assert es <= 1e-5


@pytest.mark.parametrize("n,edges,ells,seed", CASES[:2])
def test_plain_bf16_is_bounded(torch_cuda, ora, n, edges, ells, seed):
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), seed)
    bins, B, status = run(torch_cuda, dk, n, edges, ells, "bf16")
    assert status == 0
    r = ora.bispectrum(dk.astype(np.complex128), n, BOX, edges, ells)
    err = gate(B, r["B"])
    print("bf16 n=%d gate error %.3g" % (n, err))
    assert err < 0.1


def test_split_f16_close_to_fp32_path(torch_cuda):
    n = 48
    edges = linear_edges(10)
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 6)
    _, B32, _ = run(torch_cuda, dk, n, edges, (0, 2, 4), "fp32")
    _, Btc, status = run(torch_cuda, dk, n, edges, (0, 2, 4), "split_f16")
    assert status == 0
    # both within 1e-5 of the oracle (the parametrised cases), so within 2e-5 of each other
    assert gate(Btc, B32) <= 2e-5


def test_wait_limit_runs_out_and_the_plan_recovers(torch_cuda):
    """Failure path of the bounded waits, without a GPU fault: with a pipeline
    wait limit of 200 cycles the first wait for a copy runs out, the kernel
    records it in the plan's error word and returns (the context stays
    usable); with the default limit restored the same plan gives the same
    bins bit for bit and a clear error word."""
    from paper_1708_05303_gb300 import bsp

    torch = torch_cuda
    n, edges = 32, linear_edges(8)
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 5)
    d = torch.from_numpy(dk).cuda()
    est = bsp.Bispectrum(n, BOX, edges, (0, 2, 4), prec="split_f16")
    before = est.compute(d).clone()
    torch.cuda.synchronize()
    assert bsp.bsp_device_status(est.plan) == 0
    bsp.bsp_set_wait_limit(est.plan, 200)
    est.compute(d)
    torch.cuda.synchronize()            # the kernel returned; no CUDA error
    code = bsp.bsp_device_status(est.plan)
    print("error word after the short limit: %#x" % code)
    assert code != 0
    bsp.bsp_set_wait_limit(est.plan, 0)
    after = est.compute(d).clone()
    torch.cuda.synchronize()
    assert bsp.bsp_device_status(est.plan) == 0
    assert torch.equal(before, after)
    with pytest.raises(bsp.BspError):
        bsp.bsp_set_wait_limit(est.plan, -1)
    est.close()
