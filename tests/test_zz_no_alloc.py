"""The allocation-free entry point bsp_triple_sums_static against the plan
path, through the C ABI, on two calls in a row.

Callers that cannot allocate device memory (a graph under capture, a fixed
external pool) get triple sums from fixed library-owned scratch; its results
must agree with the raw sums the normal bsp_compute path produces for the
same fields, within the 1e-5 tolerance the parity tests use, and repeat
exactly.  Collected last on purpose: it runs after every other test in a
stop-at-first-failure run, and it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1708_05303_gb300.synth import FieldModel, linear_edges, make_field

pytestmark = pytest.mark.gpu


def test_static_scratch_matches_plan_path_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_05303_gb300 import build

    build.build()
    from paper_1708_05303_gb300 import bsp

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
        outs.append(T.cpu().numpy().reshape(len(ells), -1))
    ref = T_plan
    rms = np.sqrt(np.mean(ref ** 2, axis=1, keepdims=True))
    for got in outs:
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), rms)) <= 1e-5
    assert np.array_equal(outs[0], outs[1])
    with pytest.raises(bsp.BspError):
        bad = trip.copy()
        bad[0, 0] = nfields
        bsp.bsp_triple_sums_static(fields, npts, nfields, bad, T)
    est.close()
