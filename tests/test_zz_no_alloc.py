"""The allocation-free entry point bsp_triple_sums_static, through the C ABI.

Some callers cannot call cudaMalloc: a host runtime that hands out all device
memory from its own fixed pool, or an embedded caller with a hard memory
budget that must know up front every byte the library holds.  For them the
library keeps its scratch (triplet list, per-segment partial sums) in fixed
device arrays.  These tests check that entry point against the library's
normal bsp_compute path and against the oracle's triple sums, within the
1e-5 tolerance of the parity tests, on two calls in a row (the scratch keeps
the previous call's contents), on a side stream, and in the case where the
fixed partial-sum array caps the number of segments.

Collected last on purpose: in a stop-at-first-failure run every other test
has run before it; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1708_05303_gb300.synth import FieldModel, linear_edges, make_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_05303_gb300 import build

    build.build()
    from paper_1708_05303_gb300 import bsp

    return torch, bsp


def gate(got, ref):
    rms = np.sqrt(np.mean(ref ** 2))
    return np.max(np.abs(got - ref) / np.maximum(np.abs(ref), rms))


def test_static_scratch_matches_plan_path_and_oracle_twice(cuda, ora):
    torch, bsp = cuda
    n, box = 32, 1000.0
    edges = linear_edges(8)
    ells = (0, 2, 4)
    dk, _ = make_field(FieldModel(n=n, box=box, sigma_g=0.3), 4242)
    est = bsp.Bispectrum(n, box, edges, ells, prec="fp32")
    est.compute(torch.from_numpy(dk).cuda())
    T_plan = est.raw().cpu().numpy()
    nsh, npts = len(edges) - 1, n ** 3
    # FP32 plan workspace starts with the fields: slot(l) * n_shells + shell, [npts] each
    nfields = len(ells) * nsh
    trip = np.array([(li * nsh + a, b, c) for li in range(len(ells)) for (a, b, c) in est.bins], dtype=np.int32)
    fields = est.ws[: nfields * npts * 4].view(torch.float32)
    outs = []
    for _ in range(2):
        T = torch.full((len(trip),), float("nan"), dtype=torch.float64, device="cuda")
        bsp.bsp_triple_sums_static(fields, npts, nfields, trip, T)
        torch.cuda.synchronize()
        outs.append(T.cpu().numpy())
    # the oracle's compensated FP64 triple sums of the very same FP32 fields
    host = fields.cpu().numpy().reshape(nfields, npts).astype(np.float64)
    T_ora, _ = ora.sum3(list(host), trip)
    for got in outs:
        assert np.all(np.isfinite(got))
        assert gate(got.reshape(len(ells), -1), T_plan) <= 1e-5
        assert gate(got, T_ora) <= 1e-5
    assert np.array_equal(outs[0], outs[1])
    with pytest.raises(bsp.BspError):
        bad = trip.copy()
        bad[0, 0] = nfields
        bsp.bsp_triple_sums_static(fields, npts, nfields, bad, T)
    est.close()


def test_static_scratch_capped_segments_on_side_stream(cuda, ora):
    """20 000 triplets over 512 000 points: the fixed array of 2 097 152
    partial sums allows only 104 segments where the length alone would ask
    for 125, so the cap decides the split.  Run on a non-default stream,
    twice, and compare a sample of triplets with the oracle's sums."""
    torch, bsp = cuda
    npts, nfields, ntrip = 80 ** 3, 12, 20000
    rng = np.random.Generator(np.random.PCG64(77))
    host = rng.standard_normal((nfields, npts)).astype(np.float32)
    trip = rng.integers(0, nfields, size=(ntrip, 3)).astype(np.int32)
    assert (npts + 4095) // 4096 > (1 << 21) // ntrip
    fields = torch.from_numpy(host).cuda()
    side = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(side):
        for _ in range(2):
            T = torch.full((ntrip,), float("nan"), dtype=torch.float64, device="cuda")
            bsp.bsp_triple_sums_static(fields, npts, nfields, trip, T, stream=side)
            outs.append(T)
    side.synchronize()
    outs = [t.cpu().numpy() for t in outs]
    pick = rng.choice(ntrip, size=64, replace=False)
    T_ora, _ = ora.sum3(list(host.astype(np.float64)), trip[pick])
    # random fields: the sums cancel to ~sqrt(npts), so gate on the scale of the summands
    scale = np.sqrt(npts) * np.ones_like(T_ora)
    for got in outs:
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got[pick] - T_ora) / np.maximum(np.abs(T_ora), scale)) <= 1e-5
    assert np.array_equal(outs[0], outs[1])
