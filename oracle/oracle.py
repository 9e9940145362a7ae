"""FP64 CPU oracle for the FFT bispectrum-multipole estimator and its modal variant.

Regan, "An Inventory of Bispectrum Estimators for Redshift Space Distortions",
arXiv:1708.05303.  Section/equation labels below are the paper's.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may use this module.  It imports nothing
from the CUDA package and the CUDA package imports nothing from it; the two
meet only in the seeded inputs the tests hand to both.

Conventions (shared with the CUDA path by definition, not by code):

* Grid side ``n`` (even), box side ``box`` (V = box^3), k_f = 2 pi / box.
  Integer frequency per axis in C order (x, y, z), index j -> j for j < n/2,
  j - n otherwise (so index n/2 is frequency -n/2).  The line of sight is z,
  the last axis; mu = n_z / |n| (0 at the origin).
* delta(k) is continuum normalised, delta(k) = (V/n^3) sum_x delta_x e^{-ik.x},
  handed over as the half spectrum ``[n][n][n/2+1]`` (numpy rfftn layout).
* Shell a holds the modes with lo_a <= |n| < hi_a (edges in units of k_f),
  decided on the integer n^2 as lo_a*lo_a <= n^2 < hi_a*hi_a (Sec. 2 and
  Sec. 3.1 average over k +- dk/2).
* The Legendre weight of the multipole leg is w_l(mu) = (2l+1) L_l(mu)
  (Sec. 2, the definition of delta^{(l)} under Eq. PowSpecMultipole).
* Bins are (a, b, c) with a >= b >= c (shell indices); the Legendre leg is
  a, the largest side (Sec. 3.1, "with respect to the largest side").  A bin
  is valid when it holds at least one triangle.

Parity pins: tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build", "num_threads", "fft1d", "fft3d", "freq_axis", "n2_grid", "mu_grid",
    "legendre_weight", "shell_masks", "full_from_half", "real_field", "sum3",
    "brute_triangles", "candidate_triplets", "counts", "bispectrum",
    "shot_noise", "modal_q", "modal_radial", "modal_fields", "modal_triplets",
    "modal_raw", "modal_mode_order", "modal_gamma", "modal_beta", "covariance",
    "power_multipoles", "density_from_particles", "skew_spectrum", "integrated_bispectrum",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bispec_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libbispec_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C half of the oracle (gcc, -O2, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.ora_fft1d.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            lib.ora_fft3d.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            lib.ora_real_field.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_void_p, dp, dp]
            lib.ora_sum3.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long,
                                     ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p]
            lib.ora_sum3.restype = None
            lib.ora_brute.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_void_p,
                                                              ctypes.c_long, ctypes.c_void_p,
                                                              ctypes.c_long, dp, dp, dp]
            lib.ora_brute.restype = None
            lib.ora_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the C half uses (OMP_NUM_THREADS, else all cores)."""
    return int(_L().ora_num_threads())


# ----------------------------------------------------------------------------
# Discrete Fourier transforms (own code; numpy.fft is used only by the tests
# that pin these).
# ----------------------------------------------------------------------------

def fft1d(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 1-D DFT, X[k] = sum_j x[j] exp(sign 2 pi i j k / n)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    if _L().ora_fft1d(_ptr(a), a.size, int(sign)) != 0:
        raise MemoryError("ora_fft1d failed")
    return a


def fft3d(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 3-D DFT of an [n][n][n] grid (own mixed-radix code)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    n = a.shape[0]
    assert a.shape == (n, n, n)
    if _L().ora_fft3d(_ptr(a), n, int(sign)) != 0:
        raise MemoryError("ora_fft3d failed")
    return a


# ----------------------------------------------------------------------------
# Grid geometry
# ----------------------------------------------------------------------------

def freq_axis(n: int) -> np.ndarray:
    """Integer frequency of each index along one axis (index n/2 -> -n/2)."""
    j = np.arange(n, dtype=np.int64)
    return np.where(j < n // 2, j, j - n)


def n2_grid(n: int, half: bool = False) -> np.ndarray:
    """Integer |n|^2 on the full [n][n][n] grid (or the [n][n][n/2+1] half grid)."""
    f = freq_axis(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64) if half else f
    if half:
        fz = np.where(fz == n // 2, -(n // 2), fz)
    return f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2


def mu_grid(n: int, half: bool = False) -> np.ndarray:
    """mu = n_z/|n| with z the line of sight (0 at the origin)."""
    f = freq_axis(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64) if half else f
    if half:
        fz = np.where(fz == n // 2, -(n // 2), fz)
    n2 = n2_grid(n, half).astype(np.float64)
    nz = np.broadcast_to(fz[None, None, :].astype(np.float64), n2.shape)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(n2 > 0, nz / np.sqrt(n2), 0.0)
    return mu


def legendre_weight(ell: int, mu):
    """w_l(mu) = (2l+1) L_l(mu): the factor that turns delta into delta^{(l)}
    (Sec. 2 under Eq. PowSpecMultipole; Sec. 3.1 Eq. Standard_ell_Estim).
    L_0 = 1, L_2 = (3 mu^2 - 1)/2, L_4 = (35 mu^4 - 30 mu^2 + 3)/8."""
    mu = np.asarray(mu, dtype=np.float64)
    if ell == 0:
        L = np.ones_like(mu)
    elif ell == 2:
        L = (3.0 * mu ** 2 - 1.0) / 2.0
    elif ell == 4:
        L = (35.0 * mu ** 4 - 30.0 * mu ** 2 + 3.0) / 8.0
    else:
        raise ValueError("only even l in {0, 2, 4} (parity, Sec. 3.5)")
    return (2 * ell + 1) * L


def shell_masks(n: int, edges, half: bool = False):
    """Boolean shell masks lo^2 <= n^2 < hi^2 (edges in k_f units)."""
    n2 = n2_grid(n, half).astype(np.float64)
    e = [float(v) for v in edges]
    return [(n2 >= e[i] * e[i]) & (n2 < e[i + 1] * e[i + 1]) for i in range(len(e) - 1)]


def full_from_half(half: np.ndarray, n: int) -> np.ndarray:
    """Full [n][n][n] spectrum from the [n][n][n/2+1] half spectrum, made
    exactly Hermitian: the values with 0 < n_z < n/2 are taken as given and
    mirrored, delta(-n) = conj delta(n); on the n_z = 0 and n_z = n/2 planes,
    where the half spectrum holds both n and -n, the Hermitian part
    (delta(n) + conj delta(-n))/2 is used.  A real inverse transform of the
    half spectrum sees exactly this Hermitian part, so nothing the estimator
    computes changes; self-conjugate points keep their real part only."""
    h = np.asarray(half, dtype=np.complex128)
    assert h.shape == (n, n, n // 2 + 1)

    def negate(a, axis):
        # index j -> (-j) mod n along `axis`
        return np.roll(np.flip(a, axis=axis), 1, axis=axis)

    full = np.empty((n, n, n), dtype=np.complex128)
    full[:, :, : n // 2 + 1] = h
    # n_z in (n/2, n): delta(nx, ny, nz) = conj delta(-nx, -ny, n - nz)
    full[:, :, n // 2 + 1:] = np.conj(negate(negate(h, 0), 1)[:, :, 1: n // 2][:, :, ::-1])
    mirror = np.conj(negate(negate(negate(full, 0), 1), 2))
    full += mirror
    full *= 0.5
    return full


def real_field(full: np.ndarray, weight: np.ndarray) -> np.ndarray:
    """D(x) = sum_n W(n) delta(n) e^{+2 pi i n.x/n}: the real-space filtered
    field of Sec. 3.1 (D_k^{(l)} of Eq. Standard_ell_Estim up to the constant
    volume factors, which cancel against the counts).  Own FFT; returns the
    real part after checking that the imaginary part is round-off."""
    n = full.shape[0]
    spec = np.ascontiguousarray(full, dtype=np.complex128)
    w = np.ascontiguousarray(weight, dtype=np.float64)
    out = np.empty((n, n, n), dtype=np.float64)
    mi, mr = ctypes.c_double(), ctypes.c_double()
    st = _L().ora_real_field(_ptr(spec), _ptr(w), n, _ptr(out), ctypes.byref(mi), ctypes.byref(mr))
    if st != 0:
        raise MemoryError("ora_real_field failed")
    if mi.value > 1e-9 * max(mr.value, 1e-300):
        raise AssertionError("filtered field not real: max|Im| = %g vs max|Re| = %g"
                             % (mi.value, mr.value))
    return out


def sum3(fields, triples):
    """For each (i, j, k) in ``triples``: (sum_x F_i F_j F_k, sum_x (F_i F_j F_k)^2),
    compensated FP64 sums in x order (the x-integral of Eq. Standard_ell_Estim)."""
    fl = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
    npts = fl[0].size
    for f in fl:
        assert f.size == npts
    tri = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    ptrs = (ctypes.c_void_p * len(fl))(*[f.ctypes.data for f in fl])
    s = np.zeros(len(tri))
    q = np.zeros(len(tri))
    if len(tri):
        _L().ora_sum3(ptrs, _ptr(tri), len(tri), npts, _ptr(s), _ptr(q))
    return s, q


def brute_triangles(full: np.ndarray, W1, W2, W3):
    """Direct triangle sum over n1 + n2 + n3 = 0 (mod n):
    sum W1(n1) W2(n2) W3(n3) delta(n1) delta(n2) delta(n3), and the number of
    such triangles with all three weights nonzero (Eq. Bisp_ell_restrict
    aggregated over the bin; V_B of Sec. 3.1 counted on the grid)."""
    n = full.shape[0]
    spec = np.ascontiguousarray(full, dtype=np.complex128)
    W1, W2, W3 = (np.ascontiguousarray(w, dtype=np.float64) for w in (W1, W2, W3))
    i1 = np.ascontiguousarray(np.flatnonzero(W1).astype(np.int64))
    i2 = np.ascontiguousarray(np.flatnonzero(W2).astype(np.int64))
    re, im, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _L().ora_brute(_ptr(spec), _ptr(W1), _ptr(W2), _ptr(W3), n, _ptr(i1), i1.size, _ptr(i2),
                   i2.size, ctypes.byref(re), ctypes.byref(im), ctypes.byref(cnt))
    return complex(re.value, im.value), cnt.value


# ----------------------------------------------------------------------------
# Standard estimator (Sec. 3.1)
# ----------------------------------------------------------------------------

def candidate_triplets(n_shells: int):
    """All (a, b, c) with a >= b >= c, lexicographic."""
    return [(a, b, c) for a in range(n_shells) for b in range(a + 1) for c in range(b + 1)]


def counts(n: int, edges, triplets=None):
    """N_abc: the number of grid triangles n1 + n2 + n3 = 0 (mod n) with
    n1 in a, n2 in b, n3 in c -- V_B of Sec. 3.1 on the grid, "similarly
    evaluated" through unit fields I_a(x) = sum_{n in a} e^{i k.x}:
    N_abc = (1/n^3) sum_x I_a I_b I_c.  Rounded to the nearest integer."""
    masks = shell_masks(n, edges)
    ones = np.ones((n, n, n), dtype=np.complex128)
    if triplets is None:
        triplets = candidate_triplets(len(masks))
    need = sorted({s for t in triplets for s in t})
    idx = {s: i for i, s in enumerate(need)}
    I = [real_field(ones, masks[s].astype(np.float64)) for s in need]
    tri = [(idx[a], idx[b], idx[c]) for (a, b, c) in triplets]
    s, _ = sum3(I, tri)
    return np.rint(s / float(n) ** 3)


def bispectrum(delta_half: np.ndarray, n: int, box: float, edges, ells=(0, 2, 4), bins=None,
               nbar: float | None = None):
    """B^{(l)}(a, b, c) of Eq. Standard_ell_Estim for every valid bin.

    T^l_abc = sum_x F^l_a F^0_b F^0_c with F^l_a = sum_{n in a} w_l(mu) delta(n) e^{ik.x}
    equals n^3 times the triangle sum of w_l(mu_1) delta_1 delta_2 delta_3, and
    B^l = T^l / (V n^3 N_abc): the bin average of Eq. Bisp_ell_restrict.  The
    (2 pi)^3 and n^3 factors of Sec. 3.1 cancel between numerator and V_B.
    With ``nbar`` the Poisson shot noise of ``shot_noise`` is subtracted.

    Returns a dict: bins [nb,3], counts [nb], T [nl,nb], B [nl,nb],
    sumsq [nl,nb] (sum_x of the squared summand, the round-off scale)."""
    masks = shell_masks(n, edges)
    ns = len(masks)
    full = full_from_half(delta_half, n)
    if bins is None:
        cand = candidate_triplets(ns)
        cnt = counts(n, edges, cand)
        bins = [t for t, c in zip(cand, cnt) if c >= 1]
        cnt = np.array([c for c in cnt if c >= 1])
    else:
        bins = [tuple(int(v) for v in t) for t in bins]
        cnt = counts(n, edges, bins)
    mu = mu_grid(n)
    legs_a = sorted({t[0] for t in bins})
    legs_bc = sorted({s for t in bins for s in t[1:]})
    fields, key = [], {}
    for ell in ells:
        wl = legendre_weight(ell, mu)
        for a in (legs_a if ell != 0 else sorted(set(legs_a) | set(legs_bc))):
            key[(ell, a)] = len(fields)
            fields.append(real_field(full, wl * masks[a]))
    for s in legs_bc:
        if (0, s) not in key:
            key[(0, s)] = len(fields)
            fields.append(real_field(full, masks[s].astype(np.float64)))
    T = np.zeros((len(ells), len(bins)))
    Q = np.zeros((len(ells), len(bins)))
    for li, ell in enumerate(ells):
        tri = [(key[(ell, a)], key[(0, b)], key[(0, c)]) for (a, b, c) in bins]
        T[li], Q[li] = sum3(fields, tri)
    V = float(box) ** 3
    n3 = float(n) ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        B = T / (V * n3 * cnt[None, :])
    out = {"bins": np.array(bins, dtype=np.int32).reshape(-1, 3), "counts": cnt, "T": T,
           "B": B, "sumsq": Q, "ells": tuple(ells)}
    if nbar is not None:
        out["shot"] = shot_noise(full, n, box, edges, ells, bins, cnt, nbar)
        out["B_raw"] = B
        out["B"] = B - out["shot"]
    return out


def shot_noise(full: np.ndarray, n: int, box: float, edges, ells, bins, cnt, nbar: float):
    """Poisson shot noise of B^{(l)} (the paper is silent; this is the exact
    per-triangle expectation for a Poisson sample, with P_tot = |delta|^2/V):
        w_l(mu_1) [ (|d_1|^2 + |d_2|^2 + |d_3|^2)/(V nbar) - 2/nbar^2 ],
    averaged over the bin's triangles.  Each term is separable per leg, so it
    is the same contraction on the fields S^l_a (weights w_l |delta|^2 on a),
    W^l_a (w_l on a), S_b (|delta|^2 on b) and I_b (unit)."""
    masks = shell_masks(n, edges)
    mu = mu_grid(n)
    p2 = np.abs(full) ** 2
    one = np.ones_like(full)
    V = float(box) ** 3
    n3 = float(n) ** 3
    legs_bc = sorted({s for t in bins for s in t[1:]})
    fb = {}
    for s in legs_bc:
        fb[("Sb", s)] = real_field(one, p2.real * masks[s])
        fb[("Ib", s)] = real_field(one, masks[s].astype(np.float64))
    out = np.zeros((len(ells), len(bins)))
    for li, ell in enumerate(ells):
        wl = legendre_weight(ell, mu)
        fa = {}
        for a in sorted({t[0] for t in bins}):
            fa[("Sa", a)] = real_field(one, wl * p2.real * masks[a])
            fa[("Wa", a)] = real_field(one, wl * masks[a])
        fl, idx = [], {}
        for k, v in list(fa.items()) + list(fb.items()):
            idx[k] = len(fl)
            fl.append(v)
        t1 = [(idx[("Sa", a)], idx[("Ib", b)], idx[("Ib", c)]) for (a, b, c) in bins]
        t2 = [(idx[("Wa", a)], idx[("Sb", b)], idx[("Ib", c)]) for (a, b, c) in bins]
        t3 = [(idx[("Wa", a)], idx[("Ib", b)], idx[("Sb", c)]) for (a, b, c) in bins]
        t4 = [(idx[("Wa", a)], idx[("Ib", b)], idx[("Ib", c)]) for (a, b, c) in bins]
        s1, _ = sum3(fl, t1)
        s2, _ = sum3(fl, t2)
        s3, _ = sum3(fl, t3)
        s4, _ = sum3(fl, t4)
        out[li] = ((s1 + s2 + s3) / (V * nbar) - 2.0 * s4 / nbar ** 2) / (n3 * np.asarray(cnt))
    return out


# ----------------------------------------------------------------------------
# Modal estimator (Sec. 3.5)
# ----------------------------------------------------------------------------

def modal_q(p: int, k, kmin: float, kmax: float):
    """1-D mode q_p(k): the shifted Legendre polynomial P_p on [kmin, kmax],
    zero outside (the paper leaves q_n open beyond "polynomials", Eq. Qn)."""
    k = np.asarray(k, dtype=np.float64)
    t = 2.0 * (k - kmin) / (kmax - kmin) - 1.0
    inside = (k >= kmin) & (k <= kmax)
    # P_p by the three-term recurrence (Bonnet): (j+1) P_{j+1} = (2j+1) t P_j - j P_{j-1}
    p0 = np.ones_like(t)
    if p == 0:
        v = p0
    else:
        p1 = t.copy()
        for j in range(1, p):
            p0, p1 = p1, ((2 * j + 1) * t * p1 - j * p0) / (j + 1)
        v = p1
    return np.where(inside, v, 0.0)


def modal_radial(n: int, box: float, n_modes: int, kmin: float, kmax: float, pk, sqrt_k: bool = True):
    """Radial tables R_p[n^2] = q_p(k)/sqrt(k P(k)) (Eq. betaEst, the weight w
    of Sec. 3.5), or q_p/sqrt(P) with ``sqrt_k=False``; k = k_f sqrt(n^2).
    Zero at n^2 = 0.  Shape [n_modes][3 (n/2)^2 + 1]."""
    kf = 2.0 * math.pi / box
    n2 = np.arange(3 * (n // 2) ** 2 + 1, dtype=np.float64)
    k = kf * np.sqrt(n2)
    R = np.zeros((n_modes, n2.size))
    with np.errstate(divide="ignore", invalid="ignore"):
        P = np.asarray(pk(k), dtype=np.float64)
        den = np.sqrt(k * P) if sqrt_k else np.sqrt(P)
        for p in range(n_modes):
            R[p] = np.where(n2 > 0, modal_q(p, k, kmin, kmax) / den, 0.0)
    R[~np.isfinite(R)] = 0.0
    return R


def modal_fields(full: np.ndarray, n: int, R: np.ndarray, ells):
    """M^{(l)}_p(x) = sum_n e^{ik.x} R_p(|n|) w_l(mu) delta(n) (Eq. betaEst and
    its RSD form in Sec. 3.5, constant volume factors dropped)."""
    n2 = n2_grid(n)
    mu = mu_grid(n)
    out = {}
    for ell in ells:
        wl = legendre_weight(ell, mu)
        for p in range(R.shape[0]):
            out[(ell, p)] = real_field(full, wl * R[p][n2])
    return out


def modal_triplets(n_modes: int):
    """All (p, q, r) with p <= q <= r, lexicographic."""
    return [(p, q, r) for p in range(n_modes) for q in range(p, n_modes) for r in range(q, n_modes)]


def modal_raw(M: dict, ells, triplets):
    """S^l_pqr: the x-sum of Sec. 3.5's symmetrised M^{(l1)} M^{(l2)} M^{(l3)},
    l1 + l2 + l3 = l, even l_i (Eq. Bisp_ell and the beta^l expression):
      S^0 = sum_x M0_p M0_q M0_r
      S^2 = sum_x [M2_p M0_q M0_r + M2_q M0_r M0_p + M2_r M0_p M0_q]
      S^4 = sum_x [M4_p M0_q M0_r + cyc] + sum_x [M2_p M2_q M0_r + cyc]
    (the 1/6 permutation average and the sum over the leg carrying each l_i
    combine into these three-term sums)."""
    keys = list(M.keys())
    idx = {k: i for i, k in enumerate(keys)}
    fl = [M[k] for k in keys]
    out = np.zeros((len(ells), len(triplets)))
    for li, ell in enumerate(ells):
        terms = []
        if ell == 0:
            terms.append([(idx[(0, p)], idx[(0, q)], idx[(0, r)]) for (p, q, r) in triplets])
        else:
            for rot in range(3):
                tri = []
                for t in triplets:
                    p, q, r = t[rot], t[(rot + 1) % 3], t[(rot + 2) % 3]
                    tri.append((idx[(ell, p)], idx[(0, q)], idx[(0, r)]))
                terms.append(tri)
            if ell == 4:
                for rot in range(3):
                    tri = []
                    for t in triplets:
                        p, q, r = t[rot], t[(rot + 1) % 3], t[(rot + 2) % 3]
                        tri.append((idx[(2, p)], idx[(2, q)], idx[(0, r)]))
                    terms.append(tri)
        for tri in terms:
            s, _ = sum3(fl, tri)
            out[li] += s
    return out


def modal_mode_order(n_modes_1d: int, n_keep: int):
    """3-D modes n <-> (p <= q <= r), ordered by (p+q+r, p, q, r); first n_keep."""
    tr = sorted(modal_triplets(n_modes_1d), key=lambda t: (sum(t), t[0], t[1], t[2]))
    return tr[:n_keep]


def _gl(npts):
    x, w = np.polynomial.legendre.leggauss(npts)
    return x, w


def modal_gamma(modes, kmin: float, kmax: float, npts: int = 24):
    """gamma_nm = <<Q_n|Q_m>> in the 1-D form of Sec. 3.5,
    (1/8 pi^4) int_V dk1 dk2 dk3 Q_n Q_m, V the tetrapyd
    {k_i in [kmin, kmax], 2 max k_i <= sum k_i}, Q_n the symmetrised product
    of Eq. Qn.  Nested Gauss-Legendre: k1 over [|k2-k3|, k2+k3] clipped to
    [kmin, kmax], k3 split where those limits kink, k2 split where the kinks
    cross, so the integrand is polynomial on every piece (exact for
    sufficient npts)."""
    x, w = _gl(npts)
    a, b = float(kmin), float(kmax)
    pmax = max(max(t) for t in modes) + 1

    def qv(k):
        return np.stack([modal_q(p, k, a, b) for p in range(pmax)])  # [pmax, len(k)]

    bk2 = sorted({a, b, min(max((a + b) / 2, a), b), min(max((b - a) / 2, a), b),
                  min(max(2 * a, a), b), min(max(b - a, a), b)})
    K1, K2, K3, WT = [], [], [], []
    for i in range(len(bk2) - 1):
        lo2, hi2 = bk2[i], bk2[i + 1]
        if hi2 <= lo2:
            continue
        k2s = 0.5 * (hi2 - lo2) * x + 0.5 * (hi2 + lo2)
        w2s = 0.5 * (hi2 - lo2) * w
        for k2, w2 in zip(k2s, w2s):
            br = sorted({a, b} | {v for v in (b - k2, k2 - a, k2 + a) if a < v < b})
            for j in range(len(br) - 1):
                lo3, hi3 = br[j], br[j + 1]
                k3s = 0.5 * (hi3 - lo3) * x + 0.5 * (hi3 + lo3)
                w3s = 0.5 * (hi3 - lo3) * w
                for k3, w3 in zip(k3s, w3s):
                    lo1 = max(a, abs(k2 - k3))
                    hi1 = min(b, k2 + k3)
                    if hi1 <= lo1:
                        continue
                    k1s = 0.5 * (hi1 - lo1) * x + 0.5 * (hi1 + lo1)
                    w1s = 0.5 * (hi1 - lo1) * w
                    K1.append(k1s)
                    K2.append(np.full(npts, k2))
                    K3.append(np.full(npts, k3))
                    WT.append(w1s * w2 * w3)
    K1, K2, K3, WT = (np.concatenate(v) for v in (K1, K2, K3, WT))
    q1, q2, q3 = qv(K1), qv(K2), qv(K3)
    Qs = []
    for (p, q, r) in modes:
        perms = {(p, q, r), (p, r, q), (q, p, r), (q, r, p), (r, p, q), (r, q, p)}
        acc = np.zeros_like(K1)
        for (i, j, k) in [(p, q, r), (p, r, q), (q, p, r), (q, r, p), (r, p, q), (r, q, p)]:
            acc += q1[i] * q2[j] * q3[k]
        del perms
        Qs.append(acc / 6.0)
    Qs = np.stack(Qs)
    G = (Qs * WT[None, :]) @ Qs.T
    return G / (8.0 * math.pi ** 4)


def modal_beta(gamma: np.ndarray, proj: np.ndarray) -> np.ndarray:
    """beta = gamma^{-1} <<B|Q>> (Eq. betaCalc / betaEst) by Cholesky."""
    L = np.linalg.cholesky(gamma)
    y = np.linalg.solve(L, proj.T)
    return np.linalg.solve(L.T, y).T


# ----------------------------------------------------------------------------
# Covariance over mocks (the use of mocks named in Sec. 1 and Sec. 3.1)
# ----------------------------------------------------------------------------

def covariance(rows: np.ndarray) -> np.ndarray:
    """Unbiased sample covariance of the rows (mocks) in two passes:
    mean first, then centred products; divisor M - 1."""
    X = np.asarray(rows, dtype=np.float64)
    m = X.shape[0]
    mean = X.sum(axis=0) / m
    D = X - mean
    return (D.T @ D) / (m - 1)


# ----------------------------------------------------------------------------
# Power-spectrum multipoles (Sec. 2, Eq. PowSpecMultipole)
# ----------------------------------------------------------------------------

def power_multipoles(delta_half: np.ndarray, n: int, box: float, edges, ells=(0, 2, 4), nbar: float = 0.0):
    """P^(l)(k) of Eq. PowSpecMultipole on the grid: with z the line of sight
    (plane-parallel), delta^(l)(k) delta^(0)(-k) = w_l(mu) |delta(k)|^2, and
    the average over the directions of the shell is the mean over its modes,

        P^l_a = 1/(V N_a) sum_{n in shell a} w_l(mu_n) |delta(n)|^2,

    N_a the number of modes of the full grid in the shell; delta is the
    Hermitian spectrum of ``full_from_half``.  With a number density nbar
    the Poisson expectation of |delta|^2 / V, 1/nbar, is subtracted through
    its weighted shell mean: shot^l_a = (1/nbar) (1/N_a) sum_n w_l(mu_n)
    (the paper is silent on shot noise: the Poisson expectation, weighted like the signal).
    Returns dict(P, P_raw, shot [n_ell][n_shells], Nk [n_shells])."""
    V = float(box) ** 3
    full = full_from_half(delta_half, n)
    pw = np.abs(full) ** 2
    mu = mu_grid(n)
    masks = shell_masks(n, edges)
    ns = len(masks)
    P = np.zeros((len(ells), ns))
    shot = np.zeros((len(ells), ns))
    Nk = np.zeros(ns)
    for a, m in enumerate(masks):
        Nk[a] = float(m.sum())
        if Nk[a] == 0:
            continue
        for li, ell in enumerate(ells):
            w = legendre_weight(ell, mu[m])
            P[li, a] = float(np.sum(w * pw[m])) / (V * Nk[a])
            if nbar > 0:
                shot[li, a] = float(np.sum(w)) / (nbar * Nk[a])
    return dict(P=P - shot, P_raw=P, shot=shot, Nk=Nk)


# ----------------------------------------------------------------------------
# Density input stage: cloud-in-cell assignment with interlacing
# ----------------------------------------------------------------------------

def density_from_particles(pos: np.ndarray, n: int, box: float):
    """delta(k) of a particle set, the input the estimators take (the paper
    starts from a density grid; this stage follows the standard recipe the
    particle workload names):

    * cloud-in-cell weights on two grids of n^3 cells of side H = box/n:
      grid 1 with its cells at j H, grid 2 at (j + 1/2) H;
    * delta_g = count / (N_p / n^3) - 1 on each grid;
    * forward transform, continuum normalised: (V/n^3) sum_j delta_j e^{-ik.x_j}
      with x_j the cell positions, so grid 2 carries e^{-ik.(H/2)(1,1,1)};
    * delta(k) = average of the two, divided by the CIC window
      prod_a sinc^2(pi n_a / n).

    pos: [N_p][3] positions in box units, in [0, box).  Returns (half spectrum
    complex128 [n][n][n/2+1], nbar = N_p / V)."""
    pos = np.asarray(pos, dtype=np.float64)
    npart = pos.shape[0]
    V = float(box) ** 3
    out = []
    for shift in (0.0, 0.5):
        u = (pos * (n / float(box)) - shift) % n          # cell units, grid-local
        base = np.floor(u).astype(np.int64)
        frac = u - base
        grid = np.zeros(n ** 3)
        for corner in range(8):
            o = np.array([(corner >> 2) & 1, (corner >> 1) & 1, corner & 1])
            w = np.prod(np.where(o[None, :] == 1, frac, 1.0 - frac), axis=1)
            idx = ((base + o[None, :]) % n) @ np.array([n * n, n, 1])
            grid += np.bincount(idx, weights=w, minlength=n ** 3)
        d = grid.reshape(n, n, n) * (n ** 3 / npart) - 1.0
        out.append(np.fft.rfftn(d) * (V / n ** 3))
    f = freq_axis(n).astype(np.float64)
    fz = np.arange(n // 2 + 1, dtype=np.float64)
    fz[n // 2] = -(n // 2)
    phase = np.exp(-1j * np.pi / n * (f[:, None, None] + f[None, :, None] + fz[None, None, :]))
    win = (np.sinc(f / n)[:, None, None] * np.sinc(f / n)[None, :, None] * np.sinc(fz / n)[None, None, :]) ** 2
    return 0.5 * (out[0] + phase * out[1]) / win, npart / V


# ----------------------------------------------------------------------------
# Skew-spectrum multipoles (Sec. 3.3, Eq. skewspecQ with Q the convolution)
# ----------------------------------------------------------------------------

def skew_spectrum(delta_half: np.ndarray, n: int, box: float, edges, ells=(0, 2, 4)):
    """S_{*,l}(k): the direction average over shell a of [delta * delta](-k)
    delta^(l)(k), the convolution being the transform of delta(x)^2 (Sec. 3.3,
    the estimator under Eq. skewspecQ).  Normalised with 1/V like P^(l), so
    that its mean is int d^3q/(2 pi)^3 B^(l)(k, q, |k+q|):

        S^l_a = 1/(V N_a) sum_{n in a} w_l(mu_n) Re[conj Q(n) delta(n)],
        Q(n) = (V/n^3) sum_x delta_x^2 e^{-ik.x},  delta_x = (1/V) sum_n delta(n) e^{ik.x},

    delta the Hermitian spectrum with its mean mode removed (delta(0) = 0);
    no dealiasing of the square on the grid.  Returns dict(S [n_ell][n_shells], Nk)."""
    V = float(box) ** 3
    full = full_from_half(delta_half, n)
    full[0, 0, 0] = 0.0
    dx = np.real(np.fft.ifftn(full)) * (n ** 3 / V)
    Q = np.fft.fftn(dx * dx) * (V / n ** 3)
    cross = np.real(np.conj(Q) * full)
    mu = mu_grid(n)
    masks = shell_masks(n, edges)
    S = np.zeros((len(ells), len(masks)))
    Nk = np.zeros(len(masks))
    for a, m in enumerate(masks):
        Nk[a] = float(m.sum())
        if Nk[a] == 0:
            continue
        for li, ell in enumerate(ells):
            S[li, a] = float(np.sum(legendre_weight(ell, mu[m]) * cross[m])) / (V * Nk[a])
    return dict(S=S, Nk=Nk)


# ----------------------------------------------------------------------------
# Integrated bispectrum multipoles (Sec. 3.4, the estimator after
# Eq. iB_expectation, applied to the multipoles)
# ----------------------------------------------------------------------------

def integrated_bispectrum(delta_half: np.ndarray, n: int, box: float, edges, m: int, ells=(0, 2, 4)):
    """iB^(l)(k) = (1/N_s) sum_i P^(l)(k)_i dbar_i over the N_s = m^3 cubes of
    side n/m cells: delta(x) = (1/V) sum_{n != 0} delta(n) e^{ik.x} (Hermitian
    spectrum, mean removed), dbar_i its mean over cube i, P^(l)_i the
    power-spectrum multipoles of the cube's field taken as periodic (its own
    transform (V_s/n_s^3) sum_x delta_x e^{-ik.x}, no window correction), on
    the same shells in units of the parent's k_f (a cube mode n_s has
    |n| = m |n_s|).  Returns dict(iB [n_ell][n_shells], Nk per cube, dbar,
    absum = (1/N_s) sum_i |dbar_i| (1/(V_s N_a)) sum_n |w_l| |delta_s|^2, the
    size of the products the sum adds up and partly cancels)."""
    assert n % m == 0
    ns = n // m
    V = float(box) ** 3
    Vs = V / m ** 3
    full = full_from_half(delta_half, n)
    full[0, 0, 0] = 0.0
    dx = np.real(np.fft.ifftn(full)) * (n ** 3 / V)
    mu = mu_grid(ns)
    n2s = n2_grid(ns).astype(np.float64) * m * m
    e = [float(v) for v in edges]
    masks = [(n2s > 0) & (n2s >= e[a] * e[a]) & (n2s < e[a + 1] * e[a + 1]) for a in range(len(e) - 1)]
    Nk = np.array([float(mk.sum()) for mk in masks])
    iB = np.zeros((len(ells), len(masks)))
    absum = np.zeros((len(ells), len(masks)))
    dbar = np.zeros(m ** 3)
    for c in range(m ** 3):
        i, j, k = c // (m * m), (c // m) % m, c % m
        sub = dx[i * ns:(i + 1) * ns, j * ns:(j + 1) * ns, k * ns:(k + 1) * ns]
        dbar[c] = float(sub.mean())
        pw = np.abs(np.fft.fftn(sub) * (Vs / ns ** 3)) ** 2
        for a, mk in enumerate(masks):
            if Nk[a] == 0:
                continue
            for li, ell in enumerate(ells):
                w = legendre_weight(ell, mu[mk])
                iB[li, a] += dbar[c] * float(np.sum(w * pw[mk])) / (Vs * Nk[a])
                absum[li, a] += abs(dbar[c]) * float(np.sum(np.abs(w) * pw[mk])) / (Vs * Nk[a])
    return dict(iB=iB / m ** 3, Nk=Nk, dbar=dbar, absum=absum / m ** 3)
