"""The library's host-side modal helpers (Sec. 3.5) against the oracle's
independent implementations and numpy: 3-D mode ordering, radial tables,
gamma over the tetrapyd, and the Cholesky projection.  No GPU needed."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1708_05303_gb300 import build, bsp

    build.build()
    return bsp


def test_mode_order_matches_oracle(lib, ora):
    for n1, keep in [(10, 20), (50, 50), (6, 56)]:
        assert np.array_equal(lib.bsp_modal_modes(n1, keep), np.array(ora.modal_mode_order(n1, keep)))


def test_radial_table_matches_oracle(lib, ora):
    n, box = 32, 1000.0
    kf = 2 * np.pi / box
    for sqrt_k in (True, False):
        R = lib.bsp_modal_radial_powerlaw(n, box, 6, kf, 12 * kf, 2e4, -1.5, sqrt_k)
        with np.errstate(over="ignore", divide="ignore"):
            Ro = ora.modal_radial(n, box, 6, kf, 12 * kf, lambda k: 2e4 * np.power(np.maximum(k, 1e-300), -1.5),
                                  sqrt_k=sqrt_k)
        assert np.abs(R - Ro).max() <= 1e-13 * np.abs(Ro).max()


def test_gamma_matches_oracle(lib, ora):
    modes = lib.bsp_modal_modes(12, 40)
    g = lib.bsp_modal_gamma(modes, 0.00628, 0.3, 20)
    go = ora.modal_gamma([tuple(m) for m in modes], 0.00628, 0.3, 20)
    assert np.abs(g - go).max() <= 1e-12 * np.abs(go).max()
    vol = (0.3 - 0.00628) ** 3 - (0.3 - 2 * 0.00628) ** 3 / 2
    assert abs(g[0, 0] - vol / (8 * np.pi ** 4)) <= 1e-12 * g[0, 0]


def test_project_solves_gamma(lib):
    modes = lib.bsp_modal_modes(6, 12)
    g = lib.bsp_modal_gamma(modes, 0.01, 0.3, 12)
    S = np.random.default_rng(4).standard_normal((3, 12))
    beta = lib.bsp_modal_project(g, S)
    assert np.allclose(beta, np.linalg.solve(g, S.T).T, rtol=1e-9, atol=1e-12 * np.abs(beta).max())
    with pytest.raises(lib.BspError):
        lib.bsp_modal_project(-np.eye(3), np.ones((1, 3)))
