"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a direct
DFT, numpy/scipy routines, brute-force triangle sums, closed forms, a worked
example whose value follows by hand from the estimator's definition
(Sec. 3.1, Eq. Bisp_ell_restrict), the tree-level bispectrum of a local
quadratic field with the Kaiser factor (Sec. 1), a Poisson null test, and the
tetrapyd volume of Sec. 3.5.  No GPU is needed.
"""
import math

import numpy as np
import pytest

from paper_1708_05303_gb300.synth import FieldModel, delta_k_from_real, make_field

BOX = 1000.0


def direct_dft(x, sign):
    n = x.size
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n) @ x


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 15, 16, 25, 30, 49, 64, 96, 100, 160])
def test_fft1d_matches_direct_dft(ora, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        got = ora.fft1d(x, sign)
        ref = direct_dft(x, sign)
        assert np.abs(got - ref).max() <= 1e-12 * n * np.abs(x).sum() / max(n, 1) * 10 + 1e-13
    assert np.allclose(ora.fft1d(x, -1), np.fft.fft(x), rtol=0, atol=1e-11 * n)


@pytest.mark.parametrize("n", [6, 8, 12, 16])
def test_fft3d_matches_numpy(ora, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    assert np.abs(ora.fft3d(x, +1) - np.fft.ifftn(x) * n ** 3).max() < 1e-10
    assert np.abs(ora.fft3d(x, -1) - np.fft.fftn(x)).max() < 1e-10


def test_parseval_and_plane_wave(ora):
    n = 16
    x = np.zeros((n, n, n), complex)
    x[3, 5, 7] = 1.0
    X = ora.fft3d(x, -1)
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    assert np.abs(X - np.exp(-2j * np.pi * (3 * i + 5 * j + 7 * k) / n)).max() < 1e-12
    rng = np.random.default_rng(1)
    y = rng.standard_normal((n, n, n)) + 0j
    assert abs(np.sum(np.abs(ora.fft3d(y, -1)) ** 2) / n ** 3 - np.sum(np.abs(y) ** 2)) < 1e-9


def test_legendre_weight(ora):
    from scipy.special import eval_legendre

    mu = np.linspace(-1, 1, 41)
    for ell in (0, 2, 4):
        assert np.allclose(ora.legendre_weight(ell, mu), (2 * ell + 1) * eval_legendre(ell, mu),
                           atol=1e-14)
    x, w = np.polynomial.legendre.leggauss(20)
    for l1 in (0, 2, 4):
        for l2 in (0, 2, 4):
            v = np.sum(w * ora.legendre_weight(l1, x) * ora.legendre_weight(l2, x)) / 2
            # (1/2) int w_l w_m dmu = (2l+1) delta_lm
            assert abs(v - (2 * l1 + 1) * (l1 == l2)) < 1e-12
    with pytest.raises(ValueError):
        ora.legendre_weight(1, mu)


def test_grid_conventions(ora):
    n = 8
    assert list(ora.freq_axis(n)) == [0, 1, 2, 3, -4, -3, -2, -1]
    n2 = ora.n2_grid(n)
    assert n2[4, 0, 0] == 16 and n2[1, 7, 2] == 1 + 1 + 4
    mu = ora.mu_grid(n)
    assert mu[0, 0, 0] == 0.0 and mu[0, 0, 3] == 1.0 and mu[0, 0, 5] == -1.0
    assert abs(mu[1, 1, 1] - 1 / math.sqrt(3)) < 1e-15
    half = ora.n2_grid(n, half=True)
    assert half.shape == (8, 8, 5) and half[0, 0, 4] == 16
    m = ora.shell_masks(n, [1, 3, 5])
    # [1, 3): n^2 in 1..8 ; [3, 5): n^2 in 9..24
    assert m[0][1, 1, 2] and m[0][2, 2, 0] and not m[0][3, 0, 0]
    assert m[1][3, 0, 0] and m[1][4, 2, 2] and not m[1][4, 2, 3] and not m[1][0, 0, 0]


def test_full_from_half_is_hermitian_extension(ora):
    n = 10
    rng = np.random.default_rng(3)
    d = rng.standard_normal((n, n, n))
    full = ora.full_from_half(np.fft.rfftn(d), n)
    assert np.abs(full - np.fft.fftn(d)).max() < 1e-11
    # a half spectrum whose n_z = 0 plane is not Hermitian: only the Hermitian part is kept,
    # which is what a real inverse transform of the half spectrum sees
    h = np.fft.rfftn(d)
    h[1, 2, 0] += 5.0 + 3.0j
    full = ora.full_from_half(h, n)
    assert np.abs(np.fft.ifftn(full).imag).max() < 1e-12
    assert np.abs(np.fft.ifftn(full).real - np.fft.irfftn(h, s=(n, n, n), axes=(0, 1, 2))).max() < 1e-12


@pytest.mark.parametrize("n,edges", [(8, [1, 2, 3, 4]), (12, [1, 2.5, 4, 5.5, 7]),
                                     (16, [1, 3, 5, 7, 9])])
def test_fft_route_equals_brute_force_triangles(ora, n, edges):
    """T1/T2: sum_x F^l_a F_b F_c = n^3 x (direct triangle sum) to 1e-10 of
    the summand's l2 norm, and the counts exactly, for every bin and l."""
    model = FieldModel(n=n, box=BOX, sigma_g=0.3)
    dk, _ = make_field(model, 1708, dtype=np.complex128)
    r = ora.bispectrum(dk, n, BOX, edges)
    full = ora.full_from_half(dk, n)
    masks = ora.shell_masks(n, edges)
    mu = ora.mu_grid(n)
    assert len(r["bins"]) > 5
    for li, ell in enumerate((0, 2, 4)):
        wl = ora.legendre_weight(ell, mu)
        for bi, (a, b, c) in enumerate(r["bins"]):
            s, cnt = ora.brute_triangles(full, wl * masks[a], masks[b], masks[c])
            if ell == 0:
                assert cnt == r["counts"][bi]
            scale = math.sqrt(r["sumsq"][li, bi]) / n ** 3
            assert abs(s.real - r["T"][li, bi] / n ** 3) <= 1e-10 * scale
            assert abs(s.imag) <= 1e-10 * scale
            V = BOX ** 3
            nb = r["counts"][bi]
            assert abs(r["B"][li, bi] - s.real / (V * nb)) <= 1e-10 * abs(scale / (V * nb))
    # every (a >= b >= c) left out has no triangle
    cand = ora.candidate_triplets(len(masks))
    kept = {tuple(t) for t in r["bins"]}
    one = np.ones((n, n, n))
    for t in cand:
        if t not in kept:
            _, cnt = ora.brute_triangles(one + 0j, masks[t[0]], masks[t[1]], masks[t[2]])
            assert cnt == 0


def test_legendre_leg_on_any_side_equals_brute_force(ora):
    """The full-tensor reading of Sec. 3.1: with the bins (a; b >= c) for every
    assignment of the Legendre leg (not only the largest side), the oracle's
    FFT route equals the direct triangle sum with w_l on the shell a, to 1e-10
    of the summand's norm; l = 0 is the same for every assignment of one
    bin's shells, and l = 2 is not (the weighted leg matters)."""
    n, edges = 12, [1, 2.5, 4, 5.5, 7]
    dk, _ = make_field(FieldModel(n=n, box=BOX, sigma_g=0.3), 1711, dtype=np.complex128)
    sorted_bins = [tuple(int(v) for v in t) for t in ora.bispectrum(dk, n, BOX, edges, ells=(0,))["bins"]]
    full_bins = sorted({(t[k], max(t[(k + 1) % 3], t[(k + 2) % 3]), min(t[(k + 1) % 3], t[(k + 2) % 3]))
                        for t in sorted_bins for k in range(3)})
    assert any(a < b for (a, b, c) in full_bins)
    r = ora.bispectrum(dk, n, BOX, edges, bins=full_bins)
    full = ora.full_from_half(dk, n)
    masks = ora.shell_masks(n, edges)
    mu = ora.mu_grid(n)
    for li, ell in enumerate((0, 2, 4)):
        wl = ora.legendre_weight(ell, mu)
        for bi, (a, b, c) in enumerate(full_bins):
            s, _ = ora.brute_triangles(full, wl * masks[a], masks[b], masks[c])
            scale = math.sqrt(r["sumsq"][li, bi]) / n ** 3
            assert abs(s.real - r["T"][li, bi] / n ** 3) <= 1e-10 * scale
    key = {t: i for i, t in enumerate(full_bins)}
    moved = 0
    for t in sorted_bins:
        if len(set(t)) < 3:
            continue
        ia, ic = key[t], key[(t[2], t[0], t[1])]
        assert abs(r["B"][0, ia] - r["B"][0, ic]) <= 1e-10 * abs(r["B"][0, ia])
        moved += abs(r["B"][1, ia] - r["B"][1, ic]) > 1e-6 * abs(r["B"][1, ia])
    assert moved > 0


def test_thin_shell_counts(ora):
    """T3: N_abc -> 8 pi^2 k_a k_b k_c dk^3 / k_f^6 for thin, non-degenerate,
    unaliased shells (V_B of Sec. 3.1 in the continuum limit)."""
    n = 64
    one = np.ones((n, n, n), complex)
    dk = 2.0

    def unit(kc):
        return ora.real_field(one, ora.shell_masks(n, [kc - dk / 2, kc + dk / 2])[0].astype(float))

    for tri in [(9, 9, 9), (10, 8, 6), (12, 10, 9), (15, 15, 15), (14, 10, 8), (18, 12, 10)]:
        assert tri[1] + tri[2] - tri[0] >= 2 * dk and max(tri) + dk / 2 < n / 3
        I = [unit(k) for k in tri]
        s, _ = ora.sum3(I, [(0, 1, 2)])
        N = s[0] / n ** 3
        assert abs(N - round(N)) < 1e-6
        ratio = N / (8 * math.pi ** 2 * tri[0] * tri[1] * tri[2] * dk ** 3)
        assert 0.95 < ratio < 1.05, (tri, ratio)


def test_b0_permutation_symmetry(ora):
    """T4: B_0 (and the raw sum) does not depend on which leg is listed first."""
    n = 24
    model = FieldModel(n=n, box=BOX, sigma_g=0.3)
    dk, _ = make_field(model, 11, dtype=np.complex128)
    edges = [1, 3, 5, 7, 9]
    bins = [(3, 2, 1), (2, 3, 1), (1, 2, 3), (3, 1, 2), (2, 1, 3), (1, 3, 2)]
    r = ora.bispectrum(dk, n, BOX, edges, ells=(0, 2), bins=bins)
    T0 = r["T"][0]
    assert np.abs(T0 - T0[0]).max() <= 1e-12 * abs(T0[0])
    # l = 2 depends on which leg carries the Legendre weight: (3;2,1) = (3;1,2) only
    T2 = r["T"][1]
    assert abs(T2[0] - T2[3]) <= 1e-12 * abs(T2[0])
    assert abs(T2[0] - T2[1]) > 1e-6 * abs(T2[0])


def _cosine_field(n, qs):
    x = np.indices((n, n, n)).reshape(3, -1).T
    d = np.zeros(n ** 3)
    for q in qs:
        d += np.cos(2 * np.pi * (x @ np.array(q)) / n)
    return d.reshape(n, n, n)


def test_worked_example_three_cosines(ora):
    """T5: delta(x) = sum_i cos(q_i.x), q1+q2+q3 = 0, so delta(+-q_i) = V/2 and
    zero elsewhere.  By Eq. Bisp_ell_restrict the only nonzero bin is the one
    holding (|q1|,|q2|,|q3|); with the shells distinct it holds the two
    triangles (q1,q2,q3) and (-q1,-q2,-q3), so its triangle sum is
    2 (V/2)^3 w_l(mu of the largest leg)."""
    n = 16
    V = BOX ** 3
    q1, q2 = (2, 0, 1), (0, 3, 1)
    q3 = tuple(-(u + v) for u, v in zip(q1, q2))          # (-2, -3, -2)
    edges = [1, 2.5, 4, 5.5]
    # |q1|^2 = 5, |q2|^2 = 10, |q3|^2 = 17: shells 0, 1, 2
    dk = delta_k_from_real(_cosine_field(n, [q1, q2, q3]), BOX)
    r = ora.bispectrum(dk, n, BOX, edges)
    for li, ell in enumerate((0, 2, 4)):
        for bi, t in enumerate(map(tuple, r["bins"])):
            got = r["T"][li, bi] / n ** 3
            if t == (2, 1, 0):
                mu = -2 / math.sqrt(17)
                want = 2 * (V / 2) ** 3 * float(ora.legendre_weight(ell, mu))
                assert abs(got - want) <= 1e-9 * abs(V / 2) ** 3
                assert abs(r["B"][li, bi] - want / (V * r["counts"][bi])) <= 1e-9 * abs(want / V)
            else:
                assert abs(got) <= 1e-9 * (V / 2) ** 3


def test_worked_example_repeated_shell(ora):
    """T5 with two legs in one shell: q1, q2 in shell 1, q3 in shell 0.  Bin
    (1,1,0) then holds (q1,q2,q3), (q2,q1,q3) and their negatives: the
    Legendre weight is taken on the first leg only, so the sum is
    2 (V/2)^3 [w_l(mu_1) + w_l(mu_2)]."""
    n = 16
    V = BOX ** 3
    q1, q2 = (3, 0, 1), (-2, 1, -2)
    q3 = tuple(-(u + v) for u, v in zip(q1, q2))          # (-1, -1, 1)
    edges = [1, 2.5, 4]
    dk = delta_k_from_real(_cosine_field(n, [q1, q2, q3]), BOX)
    r = ora.bispectrum(dk, n, BOX, edges)
    bins = list(map(tuple, r["bins"]))
    bi = bins.index((1, 1, 0))
    for li, ell in enumerate((0, 2, 4)):
        want = 2 * (V / 2) ** 3 * float(ora.legendre_weight(ell, 1 / math.sqrt(10))
                                        + ora.legendre_weight(ell, -2 / 3))
        assert abs(r["T"][li, bi] / n ** 3 - want) <= 1e-9 * (V / 2) ** 3


@pytest.mark.slow
def test_kaiser_tree_level(ora):
    """T6: delta = g + a (g^2 - <g^2>) with the Kaiser factor (1 + f mu^2)
    per leg (Sec. 1) has, at leading order,
        B_s = prod_i (1 + f mu_i^2) 2a (P1 P2 + P2 P3 + P3 P1).
    The bin prediction sum_tri w_l(mu_1) B_s / N_tri is separable per leg and
    evaluated on weighted unit fields.  The measured mean over 32 paired (+-g)
    seeds must match it within sample variance, and nearby wrong models must not."""
    n, f, a = 32, 0.7, 0.5
    edges = [2, 4, 6, 8, 10]
    ells = (0, 2, 4)
    Bs = []
    r = None
    for s in range(32):
        acc = 0.0
        for sg in (1.0, -1.0):
            model = FieldModel(n=n, box=BOX, sigma_g=0.1, f=f, quad=a, g_sign=sg)
            dk, amp = make_field(model, 5000 + s, dtype=np.complex128)
            r = ora.bispectrum(dk, n, BOX, edges, ells)
            acc = acc + 0.5 * r["B"] / amp ** 2
        Bs.append(acc)
    Bs = np.array(Bs)
    bins, cnt = r["bins"], r["counts"]
    masks = ora.shell_masks(n, edges)
    mu = ora.mu_grid(n)
    n2 = ora.n2_grid(n)
    k = 2 * np.pi / BOX * np.sqrt(n2)
    P = np.where(n2 > 0, np.power(np.where(k > 0, k, 1.0), -1.5), 0.0)   # A = 1 (divided out)
    one = np.ones((n, n, n), complex)

    def predict(fp, ap):
        K = 1 + fp * mu ** 2
        out = np.zeros((len(ells), len(bins)))
        for li, ell in enumerate(ells):
            wl = ora.legendre_weight(ell, mu)
            fl, idx = [], {}
            for s_ in range(len(masks)):
                for key, W in (("wKP", wl * K * P), ("wK", wl * K), ("KP", K * P), ("K", K)):
                    idx[(key, s_)] = len(fl)
                    fl.append(ora.real_field(one, W * masks[s_]))
            t1 = [(idx[("wKP", A)], idx[("KP", B)], idx[("K", C)]) for A, B, C in bins]
            t2 = [(idx[("wK", A)], idx[("KP", B)], idx[("KP", C)]) for A, B, C in bins]
            t3 = [(idx[("wKP", A)], idx[("K", B)], idx[("KP", C)]) for A, B, C in bins]
            tot = sum(ora.sum3(fl, t)[0] for t in (t1, t2, t3))
            out[li] = 2 * ap * tot / (n ** 3 * cnt)
        return out

    mean = Bs.mean(0)
    err = Bs.std(0, ddof=1) / math.sqrt(len(Bs))

    def chi2(p):
        return np.mean(((mean - p) / err) ** 2, axis=1)

    good = chi2(predict(f, a))
    assert good[0] < 2.5 and good[1] < 2.5 and good[2] < 3.0, good
    for fp, ap in ((0.0, a), (0.5, a), (f, 0.45)):
        bad = chi2(predict(fp, ap))
        assert bad[0] > 3.0 * good[0], (fp, ap, bad, good)


@pytest.mark.slow
def test_shot_noise_null(ora):
    """T7: a Poisson sample of a uniform density has B = 1/nbar^2 (the third
    cumulant), and the shot-noise term removes it: the subtracted B^l is
    consistent with zero for every l, the raw B_0 is not."""
    n, lam = 16, 2.0
    edges = [1, 2.5, 4, 5.5, 7]
    raw, sub = [], []
    for s in range(48):
        rng = np.random.Generator(np.random.PCG64(900 + s))
        c = rng.poisson(lam, (n, n, n)).astype(np.float64)
        nbar_cell = c.mean()
        dk = delta_k_from_real(c / nbar_cell - 1.0, BOX)
        nbar = c.sum() / BOX ** 3
        r = ora.bispectrum(dk, n, BOX, edges, nbar=nbar)
        raw.append(r["B_raw"] * nbar ** 2)
        sub.append(r["B"] * nbar ** 2)
    raw, sub = np.array(raw), np.array(sub)
    e_sub = sub.std(0, ddof=1) / math.sqrt(len(sub))
    z = sub.mean(0) / e_sub
    assert np.mean(z ** 2) < 2.0 and np.abs(z).max() < 4.5
    z_raw0 = (raw[:, 0].mean(0) - 1.0) / (raw[:, 0].std(0, ddof=1) / math.sqrt(len(raw)))
    assert np.mean(z_raw0 ** 2) < 2.5          # raw B_0 is 1/nbar^2
    assert 0.85 < raw[:, 0].mean() < 1.15       # and clearly nonzero


def test_modal_q_is_shifted_legendre(ora):
    from scipy.special import eval_legendre

    k = np.linspace(0.0, 0.4, 101)
    for p in range(8):
        got = ora.modal_q(p, k, 0.05, 0.3)
        t = 2 * (k - 0.05) / 0.25 - 1
        want = np.where((k >= 0.05) & (k <= 0.3), eval_legendre(p, t), 0.0)
        assert np.allclose(got, want, atol=1e-12)


def test_modal_reduces_to_brute_force(ora):
    """T8: the x-space modal sum S^l_pqr / n^3 equals the Fourier-space
    definition sum over triangles of sum_{l1+l2+l3=l} prod_i w_li(mu_i) R(k_i)
    delta(k_i), averaged over the 6 permutations of (p, q, r) (Sec. 3.5,
    Eq. Bisp_ell and the beta^l expression), computed by brute force."""
    n = 12
    model = FieldModel(n=n, box=BOX, sigma_g=0.3)
    dk, amp = make_field(model, 21, dtype=np.complex128)
    full = ora.full_from_half(dk, n)
    kf = 2 * np.pi / BOX
    kmin, kmax = kf, 5.5 * kf
    R = ora.modal_radial(n, BOX, 3, kmin, kmax, lambda k: amp * np.power(np.maximum(k, 1e-30), -1.5))
    ells = (0, 2, 4)
    M = ora.modal_fields(full, n, R, ells)
    trip = ora.modal_triplets(3)
    S = ora.modal_raw(M, ells, trip)
    n2 = ora.n2_grid(n)
    mu = ora.mu_grid(n)
    tuples = {0: [(0, 0, 0)], 2: [(2, 0, 0), (0, 2, 0), (0, 0, 2)],
              4: [(4, 0, 0), (0, 4, 0), (0, 0, 4), (2, 2, 0), (2, 0, 2), (0, 2, 2)]}
    import itertools
    for li, ell in enumerate(ells):
        for ti, (p, q, r_) in enumerate(trip):
            tot = 0.0
            for perm in itertools.permutations((p, q, r_)):
                for (l1, l2, l3) in tuples[ell]:
                    W = [ora.legendre_weight(lv, mu) * R[m][n2] for lv, m in zip((l1, l2, l3), perm)]
                    s, _ = ora.brute_triangles(full, *W)
                    tot += s.real
            tot /= 6.0
            scale = abs(tot) + 1e-300
            assert abs(S[li, ti] / n ** 3 - tot) <= 1e-9 * max(scale, np.abs(S[li]).max() / n ** 3)


def test_modal_shell_indicators_reduce_to_standard(ora):
    """T8': with R_p the shell indicators, S^0_pqr is T^0 of bin (r,q,p) and
    S^2_pqr = T^2(p;q,r) + T^2(q;r,p) + T^2(r;p,q) of the standard estimator."""
    n = 16
    model = FieldModel(n=n, box=BOX, sigma_g=0.3)
    dk, _ = make_field(model, 5, dtype=np.complex128)
    full = ora.full_from_half(dk, n)
    edges = [1, 3, 5, 7]
    masks = ora.shell_masks(n, edges)
    nsq = np.arange(3 * (n // 2) ** 2 + 1, dtype=np.float64)
    R = np.stack([((nsq >= lo * lo) & (nsq < hi * hi)).astype(float) for lo, hi in zip(edges[:-1], edges[1:])])
    M = ora.modal_fields(full, n, R, (0, 2))
    trip = ora.modal_triplets(len(masks))
    S = ora.modal_raw(M, (0, 2), trip)
    bins0 = [(r_, q, p) for (p, q, r_) in trip]
    rs = ora.bispectrum(dk, n, BOX, edges, ells=(0, 2), bins=bins0)
    assert np.allclose(S[0], rs["T"][0], rtol=1e-11, atol=1e-11 * np.abs(S[0]).max())
    b1 = ora.bispectrum(dk, n, BOX, edges, ells=(2,), bins=[(p, q, r_) for (p, q, r_) in trip])
    b2 = ora.bispectrum(dk, n, BOX, edges, ells=(2,), bins=[(q, r_, p) for (p, q, r_) in trip])
    b3 = ora.bispectrum(dk, n, BOX, edges, ells=(2,), bins=[(r_, p, q) for (p, q, r_) in trip])
    want = b1["T"][0] + b2["T"][0] + b3["T"][0]
    assert np.allclose(S[1], want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_gamma_tetrapyd(ora):
    """T9: gamma_00 = Vol(tetrapyd)/(8 pi^4) with Vol = (b-a)^3 - (b-2a)^3/2
    for a <= b/2 (cube minus three corners k_i > k_j + k_l); gamma is
    symmetric positive definite; the quadrature is converged and agrees
    with a crude midpoint sum over the cube masked to the tetrapyd."""
    a, b = 0.00628, 0.3
    modes = ora.modal_mode_order(10, 20)
    g = ora.modal_gamma(modes, a, b, npts=16)
    vol = (b - a) ** 3 - (b - 2 * a) ** 3 / 2
    assert modes[0] == (0, 0, 0)
    assert abs(g[0, 0] - vol / (8 * math.pi ** 4)) <= 1e-12 * g[0, 0]
    assert np.allclose(g, g.T, rtol=0, atol=1e-15 * np.abs(g).max())
    assert np.linalg.eigvalsh(g).min() > 0
    g2 = ora.modal_gamma(modes, a, b, npts=24)
    assert np.abs(g - g2).max() <= 1e-10 * np.abs(g).max()
    m = 120
    h = (b - a) / m
    t = a + h * (np.arange(m) + 0.5)
    K1, K2, K3 = np.meshgrid(t, t, t, indexing="ij")
    inside = (2 * np.maximum(np.maximum(K1, K2), K3) <= K1 + K2 + K3)
    qs = [ora.modal_q(p, t, a, b) for p in range(10)]
    for (i, j) in [(0, 3), (2, 5), (7, 11), (19, 19)]:
        def Q(md):
            p, q, r = md
            acc = 0
            import itertools
            for (u, v, w) in itertools.permutations((p, q, r)):
                acc = acc + qs[u][:, None, None] * qs[v][None, :, None] * qs[w][None, None, :]
            return acc / 6
        crude = np.sum(Q(modes[i]) * Q(modes[j]) * inside) * h ** 3 / (8 * math.pi ** 4)
        assert abs(crude - g[i, j]) <= 0.02 * math.sqrt(g[i, i] * g[j, j]), (i, j, crude, g[i, j])


def test_modal_beta_inverts_gamma(ora):
    modes = ora.modal_mode_order(6, 10)
    g = ora.modal_gamma(modes, 0.01, 0.3, npts=12)
    beta_true = np.random.default_rng(0).standard_normal((3, len(modes)))
    proj = beta_true @ g
    assert np.allclose(ora.modal_beta(g, proj), beta_true, rtol=1e-8, atol=1e-8)


def test_covariance_matches_numpy(ora):
    X = np.random.default_rng(2).standard_normal((40, 7)) * 1e3 + 5e6
    assert np.allclose(ora.covariance(X), np.cov(X, rowvar=False), rtol=1e-9)


# ---------------------------------------------------------------------------
# Power-spectrum multipoles (Sec. 2, Eq. PowSpecMultipole)
# ---------------------------------------------------------------------------

def test_power_parseval(ora):
    """One shell holding every nonzero mode: V N P^0 = sum_n |delta(n)|^2, which
    Parseval's theorem fixes from the real field, (V^2/n^3)(sum x^2 - (sum x)^2/n^3)."""
    from paper_1708_05303_gb300.synth import delta_k_from_real

    n, box = 32, 1000.0
    x = np.random.default_rng(3).standard_normal((n, n, n)) + 0.3
    r = ora.power_multipoles(delta_k_from_real(x, box), n, box, [1, 3 ** 0.5 * n / 2 + 1])
    V = box ** 3
    assert r["Nk"][0] == n ** 3 - 1
    lhs = r["P"][0, 0] * r["Nk"][0] * V
    rhs = V * V / n ** 3 * (np.sum(x * x) - np.sum(x) ** 2 / n ** 3)
    assert abs(lhs - rhs) <= 1e-12 * rhs


def test_power_kaiser_multipoles(ora):
    """Linear field with Kaiser RSD, delta_s = (1 + f mu^2) g: the multipoles
    over a wide shell, divided by the mean linear power of its modes, approach
    the continuum Kaiser factors 1 + 2f/3 + f^2/5, 4f/3 + 4f^2/7, 8f^2/35
    (sample variance of 6 realisations at 64^3)."""
    from paper_1708_05303_gb300.synth import FieldModel, make_field

    n, box, f = 64, 1000.0, 0.7
    edges = [12, 28]
    kk = (2 * np.pi / box) * np.sqrt(ora.n2_grid(n).astype(float))
    m = ora.shell_masks(n, edges)[0]
    acc = np.zeros(3)
    for s in range(6):
        dk, amp = make_field(FieldModel(n=n, box=box, quad=0.0, f=f), 500 + s, dtype=np.complex128)
        P = ora.power_multipoles(dk, n, box, edges)["P"][:, 0]
        acc += P / np.mean(amp * kk[m] ** -1.5)
    acc /= 6
    kaiser = np.array([1 + 2 * f / 3 + f * f / 5, 4 * f / 3 + 4 * f * f / 7, 8 * f * f / 35])
    assert np.all(np.abs(acc - kaiser) <= 0.03), (acc, kaiser)


def test_power_white_noise_shot(ora):
    """White noise of variance s^2 has |delta|^2 / V = s^2 V / n^3 on every mode:
    with nbar = n^3 / (V s^2) the shot-subtracted multipoles vanish within
    sample variance, and so does the anisotropic part."""
    from paper_1708_05303_gb300.synth import delta_k_from_real

    n, box, sig = 64, 1000.0, 0.8
    x = np.random.default_rng(7).standard_normal((n, n, n)) * sig
    V = box ** 3
    nbar = n ** 3 / (V * sig * sig)
    r = ora.power_multipoles(delta_k_from_real(x, box), n, box, [4, 12, 20, 30], nbar=nbar)
    assert np.allclose(r["shot"][0], 1 / nbar)
    assert np.max(np.abs(r["P"])) * nbar <= 0.1


# ---------------------------------------------------------------------------
# Density input stage: cloud-in-cell with interlacing
# ---------------------------------------------------------------------------

def test_density_single_particle_closed_form(ora):
    """One particle on a grid node x0: grid 1 holds it in one cell, grid 2 (cells
    at half offsets) in eight with weight 1/8, so after the phase and the window
    delta(k) = V e^{-ik.x0} [1 + prod_a cos(k_a H/2)] / (2 W(k)) for k != 0."""
    n, box = 16, 1000.0
    H = box / n
    x0 = np.array([3, 5, 7]) * H
    d, nbar = ora.density_from_particles(x0[None, :], n, box)
    assert nbar == 1 / box ** 3
    f = ora.freq_axis(n).astype(float)
    fz = np.arange(n // 2 + 1, dtype=float)
    fz[n // 2] = -(n // 2)
    kx, ky, kz = [2 * np.pi / box * a for a in np.meshgrid(f, f, fz, indexing="ij")]
    W = (np.sinc(kx * H / (2 * np.pi)) * np.sinc(ky * H / (2 * np.pi)) * np.sinc(kz * H / (2 * np.pi))) ** 2
    cf = (0.5 * box ** 3 * np.exp(-1j * (kx * x0[0] + ky * x0[1] + kz * x0[2]))
          * (1 + np.cos(kx * H / 2) * np.cos(ky * H / 2) * np.cos(kz * H / 2)) / W)
    cf[0, 0, 0] = 0
    assert np.max(np.abs(d - cf)) <= 1e-12 * np.max(np.abs(cf))


def test_density_lattice_is_uniform(ora):
    """One particle at each cell centre fills both grids uniformly: delta = 0."""
    n, box = 16, 1000.0
    g = (np.arange(n) + 0.5) * (box / n)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    d, _ = ora.density_from_particles(P, n, box)
    assert np.max(np.abs(d)) <= 1e-9


def test_density_plane_wave_amplitude(ora):
    """Particles drawn from 1 + A cos(2 pi m x / L): the mode (m, 0, 0) of the
    interlaced, deconvolved delta(k) is V A / 2 within Poisson noise, and real."""
    n, box, m, A = 32, 1000.0, 3, 0.5
    rng = np.random.default_rng(1)
    x = rng.random(4_000_000) * box
    x = x[rng.random(x.size) < (1 + A * np.cos(2 * np.pi * m * x / box)) / (1 + A)][:2_000_000]
    P = np.stack([x, rng.random(x.size) * box, rng.random(x.size) * box], axis=1)
    d, _ = ora.density_from_particles(P, n, box)
    want = box ** 3 * A / 2
    assert abs(d[m, 0, 0] - want) <= 0.01 * want


# ---------------------------------------------------------------------------
# Skew-spectrum multipoles (Sec. 3.3, Eq. skewspecQ)
# ---------------------------------------------------------------------------

def test_skew_parseval(ora):
    """One shell holding every nonzero mode: V N S^0 = sum_n conj Q(n) delta(n),
    which Parseval's theorem fixes as (V^2/n^3) sum_x delta_x^3 (zero mean)."""
    from paper_1708_05303_gb300.synth import delta_k_from_real

    n, box = 16, 1000.0
    V = box ** 3
    x = np.random.default_rng(5).standard_normal((n, n, n))
    x -= x.mean()
    r = ora.skew_spectrum(delta_k_from_real(x, box), n, box, [1, 3 ** 0.5 * n / 2 + 1], ells=(0,))
    lhs = r["S"][0, 0] * V * r["Nk"][0]
    rhs = V * V / n ** 3 * np.sum(x ** 3)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_skew_brute_force_convolution(ora):
    """On a 6^3 grid the convolution Q(n) = (1/V) sum_q delta(q) delta(n - q)
    summed directly over all q (mod n) gives the same multipoles."""
    from paper_1708_05303_gb300.synth import delta_k_from_real

    n, box = 6, 1000.0
    V = box ** 3
    x = np.random.default_rng(6).standard_normal((n, n, n))
    x -= x.mean()
    dk = delta_k_from_real(x, box)
    full = ora.full_from_half(dk, n)
    full[0, 0, 0] = 0
    idx = np.arange(n)
    Q = np.zeros((n, n, n), complex)
    for a in range(n):
        for b in range(n):
            for c in range(n):
                sh = full[np.ix_((a - idx) % n, (b - idx) % n, (c - idx) % n)]
                Q[a, b, c] = np.sum(full * sh) / V
    mu = ora.mu_grid(n)
    edges = [1, 2, 3, 4.5]
    want = np.array([[np.sum(ora.legendre_weight(l, mu[m]) * np.real(np.conj(Q[m]) * full[m])) / (V * m.sum())
                      for m in ora.shell_masks(n, edges)] for l in (0, 2, 4)])
    got = ora.skew_spectrum(dk, n, box, edges)["S"]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_skew_sign_follows_the_quadratic_term(ora):
    """delta = g + b (g^2 - <g^2>): the large-scale skew spectrum has the sign
    of b (tree level: B > 0 for b > 0), and flips with it."""
    from paper_1708_05303_gb300.synth import FieldModel, make_field

    out = []
    for quad in (0.5, -0.5):
        dk, _ = make_field(FieldModel(n=32, box=1000.0, quad=quad, f=0.0, sigma_g=0.3), 77, dtype=np.complex128)
        out.append(ora.skew_spectrum(dk, 32, 1000.0, [1, 5, 9], ells=(0,))["S"][0])
    assert np.all(out[0] > 0) and np.all(out[1] < 0)


# ----------------------------------------------------------------------------
# Integrated bispectrum (Sec. 3.4)
# ----------------------------------------------------------------------------

def _cube_field(n, m, c, s, wave):
    """delta_x = c_i + s_i cos(2 pi q u / ns) on cube i, u the local coordinate
    along axis `wave[0]` with q = wave[1]."""
    ns = n // m
    ax, q = wave
    u = np.arange(ns)
    prof = np.cos(2 * np.pi * q * u / ns)
    shape = [1, 1, 1]
    shape[ax] = ns
    prof = prof.reshape(shape) * np.ones((ns, ns, ns))
    x = np.zeros((n, n, n))
    for i in range(m ** 3):
        a, b, d = i // (m * m), (i // m) % m, i % m
        x[a * ns:(a + 1) * ns, b * ns:(b + 1) * ns, d * ns:(d + 1) * ns] = c[i] + s[i] * prof
    return x


def _sub_counts(ns, m, edges):
    """Modes of the ns^3 sub-grid per shell, the shell decided on m^2 |n_s|^2
    (the sub-grid's fundamental is m parent fundamentals), by explicit loops."""
    cnt = [0] * (len(edges) - 1)
    fr = [j if j < ns // 2 else j - ns for j in range(ns)]
    for fx in fr:
        for fy in fr:
            for fz in fr:
                q = (fx * fx + fy * fy + fz * fz) * m * m
                for a in range(len(edges) - 1):
                    if q > 0 and edges[a] ** 2 <= q < edges[a + 1] ** 2:
                        cnt[a] += 1
    return np.array(cnt, dtype=np.float64)


@pytest.mark.parametrize("ax,w", [(2, (1.0, 5.0, 9.0)), (0, (1.0, -2.5, 3.375))])
def test_ib_plane_wave_closed_form(ora, ax, w):
    # per cube: mean c_i and a cosine of amplitude s_i (mu = 1 along z, 0
    # along x).  P^l_i holds the two modes +-q of |delta_s|^2 = (V_s s_i/2)^2,
    # so iB^l = mean_i(c_i s_i^2) w_l V_s / (2 N_a) in the shell of |n| = m q
    n, m, box, q = 16, 2, 500.0, 2
    rng = np.random.default_rng(11)
    c = rng.standard_normal(m ** 3) * 0.1
    c -= c.mean()
    s = 0.5 + rng.random(m ** 3)
    x = _cube_field(n, m, c, s, (ax, q))
    dk = delta_k_from_real(x, box)
    edges = [1.0, 3.0, 5.0, 7.0, 9.0]
    r = ora.integrated_bispectrum(dk, n, box, edges, m)
    Vs = box ** 3 / m ** 3
    Nk = _sub_counts(n // m, m, edges)
    np.testing.assert_allclose(r["Nk"], Nk)
    np.testing.assert_allclose(r["dbar"], c, atol=1e-13)
    a = 1   # |n| = m q = 4 lies in shell 1, [3, 5)
    want = np.zeros((3, len(edges) - 1))
    for li in range(3):
        want[li, a] = np.mean(c * s * s) * w[li] * Vs / (2 * Nk[a])
    scale = np.max(np.abs(want))
    np.testing.assert_allclose(r["iB"], want, atol=1e-12 * scale)


def test_ib_brute_force_loops(ora):
    # 4^3 grid in 2^3 cubes of side 2: sub-cube transforms and shell sums by
    # explicit loops over cubes, points and modes
    n, m, box = 4, 2, 10.0
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n, n, n))
    x -= x.mean()
    dk = delta_k_from_real(x, box)
    edges = [1.0, 2.5, 3.5, 5.0]
    ells = (0, 2, 4)
    ns, Vs = n // m, box ** 3 / m ** 3
    fr = [j if j < ns // 2 else j - ns for j in range(ns)]
    want = np.zeros((3, len(edges) - 1))
    cnt = np.zeros(len(edges) - 1)
    for i in range(m ** 3):
        a0, b0, d0 = (i // (m * m)) * ns, ((i // m) % m) * ns, (i % m) * ns
        dbar = sum(x[a0 + u, b0 + v, d0 + t] for u in range(ns) for v in range(ns) for t in range(ns)) / ns ** 3
        for kx in range(ns):
            for ky in range(ns):
                for kz in range(ns):
                    f = (fr[kx], fr[ky], fr[kz])
                    q = (f[0] ** 2 + f[1] ** 2 + f[2] ** 2) * m * m
                    sh = [a for a in range(len(edges) - 1) if q > 0 and edges[a] ** 2 <= q < edges[a + 1] ** 2]
                    if not sh:
                        continue
                    acc = 0j
                    for u in range(ns):
                        for v in range(ns):
                            for t in range(ns):
                                ph = -2j * math.pi * (kx * u + ky * v + kz * t) / ns
                                acc += x[a0 + u, b0 + v, d0 + t] * complex(math.cos(ph.imag), math.sin(ph.imag))
                    d = acc * Vs / ns ** 3
                    mu = f[2] * m / math.sqrt(q)
                    for li, ell in enumerate(ells):
                        leg = {0: 1.0, 2: 0.5 * (3 * mu * mu - 1), 4: (35 * mu ** 4 - 30 * mu * mu + 3) / 8}[ell]
                        want[li, sh[0]] += dbar * (2 * ell + 1) * leg * abs(d) ** 2 / Vs
                    if i == 0:
                        cnt[sh[0]] += 1
    want /= np.where(cnt > 0, cnt, 1)[None, :] * m ** 3
    r = ora.integrated_bispectrum(dk, n, box, edges, m)
    np.testing.assert_allclose(r["Nk"], cnt)
    np.testing.assert_allclose(r["iB"], want, rtol=1e-10, atol=1e-12 * np.max(np.abs(want)))


def test_ib_single_cube_vanishes(ora):
    # m = 1: the one sub-volume is the whole box, whose mean (the n = 0 mode)
    # is not part of delta, so every product P dbar is zero
    dk, _ = make_field(FieldModel(n=16, box=300.0, sigma_g=0.3), 2, dtype=np.complex128)
    r = ora.integrated_bispectrum(dk, 16, 300.0, [1.0, 3.0, 5.0, 7.0], 1)
    assert abs(r["dbar"][0]) < 1e-12
    assert np.max(np.abs(r["iB"])) < 1e-12 * max(1.0, np.max(np.abs(ora.power_multipoles(dk, 16, 300.0, [1.0, 3.0, 5.0, 7.0])["P"])))


def test_golden_512_counts_by_direct_enumeration():
    """The committed 512^3 oracle sample (tests/golden): its counts of the
    low-k bins equal a direct enumeration of the triangles q1 + q2 + q3 = 0
    with the legs in shells a, b, c (the shells are far below n/2, so no
    triangle wraps), so the file is tied to the definition, not only to the
    oracle run that wrote it."""
    import itertools
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "fullsize_512_64shells.json")))
    e = g["edges"]

    def modes(s):
        r = int(math.ceil(e[s + 1]))
        return [q for q in itertools.product(range(-r, r + 1), repeat=3)
                if e[s] ** 2 <= q[0] ** 2 + q[1] ** 2 + q[2] ** 2 < e[s + 1] ** 2]

    checked = 0
    for (a, b, c), cnt in zip(g["bins"], g["counts"]):
        if a > 2:
            continue
        mb, mc = modes(b), set(modes(c))
        n = 0
        for q1 in modes(a):
            for q2 in mb:
                if (-q1[0] - q2[0], -q1[1] - q2[1], -q1[2] - q2[2]) in mc:
                    n += 1
        assert n == cnt, ((a, b, c), n, cnt)
        checked += 1
    assert checked >= 8
