"""Pins for the FP64 CPU oracle: each test checks it against something other
than itself (brute-force least squares, closed forms, numpy's FFT, dense
matrices built with numpy.exp, the paper's Table I)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2205_02646_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# --- independent numpy helpers (no oracle code) ---------------------------
def three_quarter_pixels(codes):
    """Window coordinates of the transparent sub-pixels of each L-pixel;
    codes[pm, qm] in 0..3 (opaque quadrant) or 255 (absent)."""
    L = codes.shape[0]
    pix = []
    for pm in range(L):
        for qm in range(L):
            c = int(codes[pm, qm])
            if c == 255:
                continue
            pix.append([(2 * pm + a, 2 * qm + b) for a in (0, 1) for b in (0, 1) if 2 * a + b != c])
    return pix


def dense_M(pixels, W):
    """M[m, k] = sum over the pixels of m of exp(2 pi j (eta k1 + gamma k2) / W)."""
    k1, k2 = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    M = np.zeros((len(pixels), W * W), complex)
    for m, px in enumerate(pixels):
        for e, g in px:
            M[m] += np.exp(2j * np.pi * (e * k1 + g * k2) / W).ravel()
    return M


def mirror(k, W):
    return ((-(k // W)) % W) * W + ((-(k % W)) % W)


def rng(seed):
    return np.random.default_rng(seed)


# --- Eq. 1 ----------------------------------------------------------------
def test_measure_hand_and_independent():
    f = np.arange(16, dtype=float).reshape(4, 4)
    mask = np.array([[0, 1], [2, 3]], np.uint8)
    y = oracle.measure(f, mask)
    # footprint (0,0) = [0,1;4,5] minus TL (0) ; (0,1) = [2,3;6,7] minus TR (3)
    # (1,0) = [8,9;12,13] minus BL (12) ; (1,1) = [10,11;14,15] minus BR (15)
    assert y.tolist() == [[10.0, 15.0], [30.0, 35.0]]
    g = rng(1).random((64, 48))
    m = synth.random_mask(32, 24, 3)
    np.testing.assert_allclose(oracle.measure(g, m), synth.measure(g, m), rtol=0, atol=1e-13)


# --- Eq. 10 argmax and Eq. 16 step against brute-force least squares ------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_greedy_step_is_bruteforce_weighted_least_squares(seed):
    W, L = 8, 4
    r0 = rng(seed)
    codes = r0.integers(0, 4, (L, L)).astype(np.uint8)
    if seed == 2:
        codes[0, :] = 255                      # a clipped window
    pix = three_quarter_pixels(codes)
    w = r0.uniform(0.1, 1.0, len(pix))
    y = r0.uniform(0.0, 3.0, len(pix))
    qt = r0.uniform(0.2, 1.0, W * W)
    gam = 0.7
    nu = 10
    p = oracle.Params(window=W, nu_max=nu, gamma_odc=gam, q_mode=2, q_table=qt)
    out = oracle.window_solve(pix, w, y, p)
    M = dense_M(pix, W)
    sw = np.sqrt(w)
    c = np.zeros(W * W, complex)
    for it in range(nu):
        r = y - M @ c                                   # residual from scratch
        e0 = np.sum(w * np.abs(r) ** 2)
        gain = np.zeros(W * W)
        dk = np.zeros(W * W, complex)
        for k in range(W * W):
            sol, *_ = np.linalg.lstsq((sw * M[:, k])[:, None], sw * r, rcond=None)
            dk[k] = sol[0]
            gain[k] = qt[k] * (e0 - np.sum(w * np.abs(r - dk[k] * M[:, k]) ** 2))
        k = out["sel"][it]
        assert gain[k] >= gain.max() * (1 - 1e-9), (it, k, int(np.argmax(gain)))
        np.testing.assert_allclose(out["dc"][it] / gam, dk[k], rtol=1e-9, atol=1e-12)
        c[k] += gam * dk[k]
    np.testing.assert_allclose(out["c"].ravel(), c, rtol=1e-9, atol=1e-12)


def test_energy_identity_and_monotone():
    W, L = 16, 8
    r0 = rng(5)
    codes = r0.integers(0, 4, (L, L)).astype(np.uint8)
    pix = three_quarter_pixels(codes)
    w = r0.uniform(0.05, 1.0, len(pix))
    y = r0.uniform(0.0, 3.0, len(pix))
    for gam in (0.3, 1.0, 1.6):
        p = oracle.Params(window=W, nu_max=25, gamma_odc=gam)
        out = oracle.window_solve(pix, w, y, p)
        M = dense_M(pix, W)
        D = np.sum(w[:, None] * np.abs(M) ** 2, axis=0)
        c = np.zeros(W * W, complex)
        E = [np.sum(w * y ** 2)]
        for it in range(25):
            c[out["sel"][it]] += out["dc"][it]
            E.append(np.sum(w * np.abs(y - M @ c) ** 2))
        E = np.array(E)
        np.testing.assert_allclose(out["energy"], E, rtol=1e-10, atol=1e-12)
        assert np.all(np.diff(E) <= 1e-12 * E[0])
        d = out["dc"] / gam
        drop = (2 * gam - gam ** 2) * D[out["sel"]] * np.abs(d) ** 2
        np.testing.assert_allclose(E[:-1] - E[1:], drop, rtol=1e-8, atol=1e-12 * E[0])


# --- closed forms ----------------------------------------------------------
@pytest.mark.parametrize("W,k0", [(8, (3, 5)), (32, (7, 19))])
def test_single_atom_recovered_in_one_step(W, k0):
    L = W // 2
    codes = rng(W).integers(0, 4, (L, L)).astype(np.uint8)
    pix = three_quarter_pixels(codes)
    w = 0.7 ** rng(W + 1).uniform(0, 20, len(pix))
    M = dense_M(pix, W)
    k = k0[0] * W + k0[1]
    y = M[:, k]                                   # measurement of f = Phi_k0
    p = oracle.Params(window=W, nu_max=1, gamma_odc=1.0, q_mode=1)
    out = oracle.window_solve(pix, w, y, p)
    assert out["sel"][0] == k
    assert abs(out["dc"][0] - 1.0) < 1e-12
    assert np.max(np.abs(out["r"])) < 1e-11


def test_identity_measurement_is_fft_and_recovers_sparse_exactly():
    W = 8
    pix = [[(e, g)] for e in range(W) for g in range(W)]
    w = np.ones(W * W)
    r0 = rng(11)
    ks = r0.choice(W * W, 5, replace=False)
    coef = (r0.uniform(0.5, 2.0, 5) * np.exp(2j * np.pi * r0.random(5)))
    k1, k2 = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    img = np.zeros((W, W), complex)
    for k, a in zip(ks, coef):
        img += a * np.exp(2j * np.pi * ((k // W) * k1 + (k % W) * k2) / W)
    y = img.ravel()
    p1 = oracle.Params(window=W, nu_max=1, gamma_odc=1.0, q_mode=1)
    out1 = oracle.window_solve(pix, w, y, p1)
    F = np.fft.fft2(img).ravel()                   # projected residual R^0
    kstar = int(np.argmax(np.abs(F)))
    assert out1["sel"][0] == kstar
    np.testing.assert_allclose(out1["dc"][0], F[kstar] / W ** 2, rtol=1e-12)
    p5 = oracle.Params(window=W, nu_max=5, gamma_odc=1.0, q_mode=1)
    out5 = oracle.window_solve(pix, w, y, p5)
    truth = np.zeros(W * W, complex)
    truth[ks] = coef
    np.testing.assert_allclose(out5["c"].ravel(), truth, atol=1e-12)
    assert sorted(out5["sel"].tolist()) == sorted(ks.tolist())


def test_measurement_consistency_real_part_of_residual():
    f, mask, y = synth.workload("rljsde_64x64")
    W, off = 32, 14
    bi, bj = 6, 9
    p0, q0 = (4 * bi - off) // 2, (4 * bj - off) // 2
    codes = mask[p0:p0 + 16, q0:q0 + 16]
    pix = three_quarter_pixels(codes)
    ym = y[p0:p0 + 16, q0:q0 + 16].astype(np.float64).ravel()
    wm = 0.7 ** np.hypot(*np.meshgrid(2 * np.arange(16) - 15.0, 2 * np.arange(16) - 15.0, indexing="ij")).ravel()
    p = oracle.Params(nu_max=30)
    out = oracle.window_solve(pix, wm, ym, p)
    k1, k2 = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    eta, gam = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    model = np.zeros((W, W), complex)
    for k in np.nonzero(out["c"].ravel())[0]:
        model += out["c"].ravel()[k] * np.exp(2j * np.pi * ((k // W) * eta + (k % W) * gam) / W)
    re_int = np.array([sum(model[e, g].real for e, g in px) for px in pix])
    np.testing.assert_allclose(out["r"].real, ym - re_int, atol=1e-10)
    assert out["energy"][-1] < out["energy"][0]


# --- Eqs. 12-14 tables against dense matrices -------------------------------
@pytest.mark.parametrize("W", [8, 32])
def test_tables_equal_dense_gram(W):
    L = W // 2
    r0 = rng(21 + W)
    codes = r0.integers(0, 4, (L, L)).astype(np.uint8)
    codes[:, :2] = 255
    pix = three_quarter_pixels(codes)
    w = r0.uniform(0.01, 1.0, len(pix))
    B, C, D = oracle.window_tables(pix, w, W)
    M = dense_M(pix, W)
    np.testing.assert_allclose(B, w[:, None] * np.conj(M), atol=1e-12)
    Cd = np.conj(M).T @ (w[:, None] * M)
    np.testing.assert_allclose(C, Cd, atol=1e-10 * np.abs(Cd).max())
    np.testing.assert_allclose(D, np.real(np.diag(Cd)), rtol=1e-12)
    np.testing.assert_allclose(C, np.conj(C.T), atol=1e-12 * np.abs(Cd).max())
    assert np.all(np.abs(C) ** 2 <= np.outer(D, D) * (1 + 1e-10) + 1e-20)


# --- invariances -----------------------------------------------------------
def test_invariances():
    W, L = 16, 8
    r0 = rng(31)
    codes = r0.integers(0, 4, (L, L)).astype(np.uint8)
    pix = three_quarter_pixels(codes)
    w = r0.uniform(0.05, 1.0, len(pix))
    y = r0.uniform(0.0, 3.0, len(pix))
    p = oracle.Params(window=W, nu_max=20)
    base = oracle.window_solve(pix, w, y, p)
    # scaling A and y together: scale y (A enters linearly) -> c scales
    sc = oracle.window_solve(pix, w, 3.7 * y, p)
    assert (sc["sel"] == base["sel"]).all()
    np.testing.assert_allclose(sc["c"], 3.7 * base["c"], rtol=1e-10, atol=1e-13)
    # scaling w leaves everything unchanged
    sw = oracle.window_solve(pix, 5.0 * w, y, p)
    assert (sw["sel"] == base["sel"]).all()
    np.testing.assert_allclose(sw["c"], base["c"], rtol=1e-10, atol=1e-13)
    # moving Phi's phase origin by (1, 2) pixels: c_k picks up exp(-2 pi j (k1 + 2 k2) / W)
    pix_s = [[(e + 1, g + 2) for e, g in px] for px in pix]
    sh = oracle.window_solve(pix_s, w, y, p)
    assert (sh["sel"] == base["sel"]).all()
    k1, k2 = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    np.testing.assert_allclose(sh["c"], base["c"] * np.exp(-2j * np.pi * (k1 + 2 * k2) / W),
                               atol=1e-11)


def test_structural_conjugate_tie_goes_to_lower_index():
    W, L = 32, 16
    r0 = rng(41)
    codes = r0.integers(0, 4, (L, L)).astype(np.uint8)
    pix = three_quarter_pixels(codes)
    w = r0.uniform(0.05, 1.0, len(pix))
    y = r0.uniform(-1.0, 1.0, len(pix))      # zero mean: DC (its own mirror) loses
    out = oracle.window_solve(pix, w, y, oracle.Params(nu_max=3))
    k = int(out["sel"][0])
    assert mirror(k, W) != k
    assert out["gap"][0] == 0.0              # real y: R(-k) = conj R(k) exactly
    assert k < mirror(k, W)


def test_argmax_takes_binary32_rounded_scores():
    """Reading of Eqs. 10-11: the argmax compares scores rounded to binary32
    (the precision of the paper's complex64 tables), lowest index on ties.
    Identity measurement of two unit atoms: both project to W^2 exactly, so
    their scores are q_k * W^2.  A frequency weight 2^-40 above 1 on the
    higher index wins in FP64 but rounds to the same binary32 value, so the
    lower index must win; 2^-20 above 1 survives the rounding and must win."""
    W = 8
    pix = [[(e, g)] for e in range(W) for g in range(W)]
    w = np.ones(W * W)
    k1, k2 = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    lo, hi = 1 * W + 2, 5 * W + 3                        # not each other's mirror
    assert mirror(lo, W) != hi
    atom = lambda k: np.exp(2j * np.pi * ((k // W) * k1 + (k % W) * k2) / W).ravel()
    y = atom(lo) + atom(hi)
    for bump, want in ((2.0 ** -40, lo), (2.0 ** -20, hi)):
        q = np.full(W * W, 0.5)
        q[lo], q[hi] = 1.0, 1.0 + bump
        out = oracle.window_solve(pix, w, y, oracle.Params(window=W, nu_max=1, gamma_odc=1.0, q_mode=2, q_table=q))
        assert out["sel"][0] == want, (bump, out["sel"][0])
    # the FP64 gap the oracle reports still sees the 2^-40 difference
    q = np.full(W * W, 0.5)
    q[lo], q[hi] = 1.0, 1.0 + 2.0 ** -40
    out = oracle.window_solve(pix, w, y, oracle.Params(window=W, nu_max=1, gamma_odc=1.0, q_mode=2, q_table=q))
    assert out["gap"][0] < 1e-10


# --- image-level: direct == recurrent, local-mask counts (Table I) ----------
def test_direct_equals_recurrent_w16_full_image():
    f, mask, y = synth.workload("rljsde_64x64")
    p = oracle.Params(window=16, nu_max=60)
    a, ta = oracle.reconstruct(y, mask, p, trace=True)
    b, tb = oracle.reconstruct(y, mask, p, recurrent=True, trace=True)
    assert (ta["sel"] == tb["sel"]).all()
    assert np.max(np.abs(a - b)) <= 1e-10


@pytest.mark.slow
def test_direct_equals_recurrent_w32_blocks():
    f, mask, y = synth.workload("rljsde_64x64")
    blocks = [0, 1, 17, 34, 51, 68, 85, 102, 119, 136, 150, 255, 120, 121, 136 + 16, 136 + 18]
    p = oracle.Params(nu_max=100)
    a, ta = oracle.reconstruct(y, mask, p, blocks=blocks, trace=True)
    b, tb = oracle.reconstruct(y, mask, p, blocks=blocks, recurrent=True, trace=True)
    assert (ta["sel"] == tb["sel"]).all()
    ok = ~np.isnan(a)
    assert ok.sum() == 16 * len(set(blocks))
    assert np.max(np.abs(a[ok] - b[ok])) <= 1e-10


def test_local_mask_counts_match_table1_and_closed_forms():
    with open(os.path.join(HERE, "golden", "table1_memory.json")) as fh:
        g = json.load(fh)
    p = oracle.Params()
    m16 = synth.recurrent_mask(128, 128, g["period_hr_px"] // 2, 5)
    n_all, n_int = oracle.count_local_masks(m16, p)
    assert n_int == g["local_masks"] == 64
    K, nm = g["window"] ** 2, (g["window"] // 2) ** 2
    mb = lambda n: n * 8 / 1e6
    assert abs(mb(n_int * nm * K) - g["B_MB"]) / g["B_MB"] < 5e-3
    assert abs(mb(n_int * K * K) - g["C_MB"]) / g["C_MB"] < 5e-3
    assert abs(round(mb(n_int * K), 1) - g["D_MB"]) < 1e-9
    # closed forms: (P_HR / gcd(P_HR, B))^2 interior masks, (2 + 8)^2 in all for
    # a 4x4 LR tile (4 top- and 4 bottom-clipped positions per axis)
    m4 = synth.recurrent_mask(32, 32, 4, 8)
    assert oracle.count_local_masks(m4, p) == (100, 4)
    m8 = synth.recurrent_mask(96, 96, 8, 8)
    assert oracle.count_local_masks(m8, p)[1] == 16


def test_mirror_and_transpose_symmetry_pin_window_geometry():
    """Flipping the sensor left-right (or transposing it) must flip (or
    transpose) the reconstruction: pins the window placement, the block copy
    and the centring of the isotropic weight on the target block."""
    f, mask, y = synth.workload("rljsde_64x64")
    p = oracle.Params(nu_max=40)
    y = y.astype(np.float64)
    hr = oracle.reconstruct(y, mask, p)
    flip = oracle.reconstruct(np.ascontiguousarray(y[:, ::-1]),
                              np.ascontiguousarray(mask[:, ::-1] ^ 1), p)
    assert np.max(np.abs(flip[:, ::-1] - hr)) < 1e-9
    swap = np.array([0, 2, 1, 3], np.uint8)
    tr = oracle.reconstruct(np.ascontiguousarray(y.T), np.ascontiguousarray(swap[mask.T]), p)
    assert np.max(np.abs(tr.T - hr)) < 1e-9


def test_frequency_weight_reading_properties():
    for W in (8, 16, 32):
        q = oracle.frequency_weight(oracle.Params(window=W))
        assert q[0, 0] == 1.0
        k = np.arange(W)
        kt = np.where(k <= W // 2, k, k - W)
        rad = np.hypot(*np.meshgrid(kt, kt, indexing="ij"))
        assert np.array_equal(q, q[(-k) % W][:, (-k) % W])          # q(-k) = q(k)
        assert np.array_equal(q, q.T)
        order = np.argsort(rad.ravel(), kind="stable")
        assert np.all(np.diff(q.ravel()[order]) <= 1e-15)          # non-increasing in |k|
        zero = np.argwhere(q < 1e-12)
        assert zero.tolist() == [[W // 2, W // 2]]
        assert np.all(q >= 0.0)


# --- other sensor layouts: per-pixel apertures (Sec. I) ----------------------
def aperture_pixels(codes):
    """Window coordinates of the transparent sub-pixels of each L-pixel with
    aperture code in 1..15 (bit 2 * dy + dx); 0 and 255 hold no measurement."""
    L = codes.shape[0]
    pix = []
    for pm in range(L):
        for qm in range(L):
            c = int(codes[pm, qm])
            if c == 255 or c == 0:
                continue
            pix.append([(2 * pm + a, 2 * qm + b) for a in (0, 1) for b in (0, 1) if (c >> (2 * a + b)) & 1])
    return pix


def test_measure_aperture_layout():
    f = np.arange(16, dtype=float).reshape(4, 4)
    mask = np.array([[1, 6], [15, 0]], np.uint8)
    # (0,0): TL only = 0; (0,1): TR 3 + BL 6; (1,0): all four; (1,1): nothing
    assert oracle.measure(f, mask, oracle.LAYOUT_APERTURE).tolist() == [[0.0, 9.0], [42.0, 0.0]]
    g = rng(2).random((64, 48))
    m = synth.random_mask(32, 24, 4)
    np.testing.assert_array_equal(oracle.measure(g, synth.apertures_of(m), 1), oracle.measure(g, m))
    a = synth.aperture_mask(32, 24, 0, 5, synth.APERTURE_SETS["all"])
    np.testing.assert_allclose(oracle.measure(g, a, 1), synth.measure(g, a, 1), rtol=0, atol=1e-13)
    with pytest.raises(RuntimeError):
        oracle.measure(g, np.full((32, 24), 4, np.uint8))
    with pytest.raises(RuntimeError):
        oracle.measure(g, np.full((32, 24), 16, np.uint8), 1)


def test_three_quarter_apertures_equal_opaque_codes():
    f, mask, y = synth.workload("rljsde_64x64")
    y = y.astype(np.float64)
    for rec in (False, True):
        p0 = oracle.Params(window=16, nu_max=40)
        p1 = oracle.Params(window=16, nu_max=40, layout=oracle.LAYOUT_APERTURE)
        a, ta = oracle.reconstruct(y, mask, p0, recurrent=rec, trace=True)
        b, tb = oracle.reconstruct(y, synth.apertures_of(mask), p1, recurrent=rec, trace=True)
        assert np.array_equal(ta["sel"], tb["sel"])
        assert np.array_equal(a, b)


def _uniform_window_case(code, seed):
    """24 x 24 LR image with one aperture code everywhere, block (5, 5) whose
    window (LR rows / cols 3..18) lies inside; w = 1, q = 1, gamma = 1."""
    y = rng(seed).uniform(0.0, 2.0, (24, 24))
    mask = np.full((24, 24), code, np.uint8)
    p = oracle.Params(nu_max=256, gamma_odc=1.0, rho_decay=1.0, q_mode=1, layout=oracle.LAYOUT_APERTURE)
    F = np.fft.fft2(y[3:19, 3:19])           # F[kap] = sum y exp(-2 pi i (p kap1 + q kap2) / 16)
    return y, mask, p, F, 5 * 12 + 5


def _check_fft_closed_form(hr, tr, F, h):
    """Quarter sampling (h = 1) and the full aperture: every candidate
    aliases with k mod 16 and, with w = q = 1, ties with its aliases; the
    lowest index kap in [0, 16)^2 wins, delta = F[kap] / (256 h(kap)), and
    after 256 iterations the model is sum_kap F[kap] / (256 h(kap)) Phi_kap."""
    sel = tr["sel"][0]
    kap = np.stack([sel // 32, sel % 32], 1)
    assert np.all(kap < 16)
    assert sorted((kap[:, 0] * 16 + kap[:, 1]).tolist()) == list(range(256))
    A = np.abs(F) ** 2
    k0 = kap[0]
    assert A[k0[0], k0[1]] >= A.max() * (1 - 1e-12)
    np.testing.assert_allclose(tr["dc"][0][0], F[k0[0], k0[1]] / (256 * h[k0[0], k0[1]]), rtol=1e-12)
    c = F / (256 * h)
    e = np.arange(14, 18)
    k = np.arange(16)
    ph = np.exp(2j * np.pi * np.outer(e, k) / 32)            # exp(2 pi i eta kap / 32)
    model = (ph @ c @ ph.T).real                             # Eq. 18 on the block
    np.testing.assert_allclose(hr[20:24, 20:24], model, atol=1e-10)


@pytest.mark.parametrize("recurrent", [False, True])
def test_quarter_sampling_reduces_to_fft2(recurrent):
    y, mask, p, F, b = _uniform_window_case(1, 61)
    hr, tr = oracle.reconstruct(y, mask, p, blocks=[b], recurrent=recurrent, trace=True)
    _check_fft_closed_form(hr, tr, F, np.ones((16, 16)))
    # the model interpolates the measured sub-pixels exactly
    np.testing.assert_allclose(hr[20:24:2, 20:24:2], y[10:12, 10:12], atol=1e-10)


def test_full_aperture_reduces_to_fft2_and_hides_nyquist():
    y, mask, p, F, b = _uniform_window_case(15, 62)
    hr, tr = oracle.reconstruct(y, mask, p, blocks=[b], trace=True)
    k = np.arange(16)
    e = np.exp(2j * np.pi * k / 32)
    h = np.outer(1 + e, 1 + e)                               # (1 + w^k1)(1 + w^k2)
    _check_fft_closed_form(hr, tr, F, h)
    # the 2x2 box sums of the model reproduce the measurements
    blk = hr[20:24, 20:24]
    np.testing.assert_allclose(blk.reshape(2, 2, 2, 2).sum(axis=(1, 3)), y[10:12, 10:12], atol=1e-10)


def test_mixed_apertures_direct_equals_recurrent_and_skip_unobservable():
    W = 16
    f = synth.image(64, 64, 32, 4, 70)
    mask = synth.aperture_mask(32, 32, 4, 71, synth.APERTURE_SETS["all"])
    y = synth.measure(f, mask, 1)
    p = oracle.Params(window=W, nu_max=40, layout=oracle.LAYOUT_APERTURE)
    a, ta = oracle.reconstruct(y, mask, p, trace=True)
    b, tb = oracle.reconstruct(y, mask, p, recurrent=True, trace=True)
    assert np.array_equal(ta["sel"], tb["sel"])
    assert np.max(np.abs(a - b)) <= 1e-10
    # one window of vertical-pair and full apertures: the candidates whose
    # atom is zero on all measurements (k1 = W/2; dense numpy check) are never
    # selected, and the residual stays consistent with the model (Eq. 7)
    codes = synth.aperture_mask(8, 8, 0, 72, (5, 15))
    pix = aperture_pixels(codes)
    M = dense_M(pix, W)
    dead = np.all(np.abs(M) < 1e-9, axis=0)
    assert dead.sum() > 0
    ym = rng(73).uniform(0.0, 2.0, len(pix))
    wm = rng(74).uniform(0.1, 1.0, len(pix))
    out = oracle.window_solve(pix, wm, ym, oracle.Params(window=W, nu_max=60))
    assert not dead[out["sel"]].any()
    model = dense_M([[(e, g)] for e in range(W) for g in range(W)], W) @ out["c"].ravel()
    re_int = np.array([sum(model[e * W + g].real for e, g in px) for px in pix])
    np.testing.assert_allclose(out["r"].real, ym - re_int, atol=1e-10)
    assert np.all(np.diff(out["energy"]) <= 1e-12)


def test_transpose_symmetric_apertures_make_identical_atoms():
    """Apertures symmetric under transposition see candidates (k1, k2) and
    (k2, k1) with k1 - k2 = 16 through identical atoms (dense numpy check);
    the oracle then meets exact ties, which it breaks to the lower index."""
    W = 32
    codes = synth.aperture_mask(16, 16, 4, 80, synth.APERTURE_SETS["symmetric"])
    M = dense_M(aperture_pixels(codes), W)
    for k1 in range(W):
        k2 = (k1 - 16) % W
        np.testing.assert_allclose(M[:, k1 * W + k2], M[:, k2 * W + k1], atol=1e-9)
    codes = synth.aperture_mask(16, 16, 4, 81, synth.APERTURE_SETS["mixed"])
    M = dense_M(aperture_pixels(codes), W)
    assert np.abs(M[:, 26 * W + 10] - M[:, 10 * W + 26]).max() > 1e-3


# --- conjugate-pair update (pairs=1), the frequency selective variant -------
def _three_quarter_window(seed, W=16):
    L = W // 2
    r0 = rng(seed)
    codes = r0.integers(0, 4, (L, L)).astype(np.uint8)
    pix = three_quarter_pixels(codes)
    return pix, r0.uniform(0.05, 1.0, len(pix)), r0.uniform(0.0, 3.0, len(pix))


def test_pairs_keep_residual_and_model_real():
    W = 16
    pix, w, y = _three_quarter_window(90, W)
    out = oracle.window_solve(pix, w, y, oracle.Params(window=W, nu_max=30, pairs=1))
    assert np.all(out["r"].imag == 0.0)
    c = out["c"]
    k = np.arange(W)
    np.testing.assert_array_equal(c[(-k) % W][:, (-k) % W], np.conj(c))
    sel = out["sel"]
    assert np.all(sel <= mirror(sel, W))                    # half-plane representatives
    # with a q that is not symmetric the mirror scores differ; the argmax
    # still only looks at the representatives
    qt = rng(93).uniform(0.1, 1.0, W * W)
    oq = oracle.window_solve(pix, w, y, oracle.Params(window=W, nu_max=30, pairs=1, q_mode=2, q_table=qt))
    assert np.all(oq["sel"] <= mirror(oq["sel"], W))
    # the model is real on the whole window
    eta = np.arange(W)
    ph = np.exp(2j * np.pi * np.outer(eta, k) / W)
    assert np.abs((ph @ c @ ph.T).imag).max() < 1e-12
    # measurement consistency (Eq. 7) with the pair updates
    model = (ph @ c @ ph.T).real
    re_int = np.array([sum(model[e, g] for e, g in px) for px in pix])
    np.testing.assert_allclose(out["r"].real, y - re_int, atol=1e-10)


@pytest.mark.parametrize("gam", [0.3, 0.5, 1.0])
def test_pairs_energy_non_increasing(gam):
    """For a real residual r, the pair step v = 2 Re(gamma delta a_k) gives
    E' - E = -4 gamma |delta|^2 D_k + |v|_w^2 <= -4 gamma (1 - gamma) |delta|^2 D_k."""
    W = 16
    pix, w, y = _three_quarter_window(91, W)
    out = oracle.window_solve(pix, w, y, oracle.Params(window=W, nu_max=40, gamma_odc=gam, pairs=1))
    e = out["energy"]
    assert np.all(np.diff(e) <= 1e-12 * e[0])
    # the bound, checked step by step with dense numpy atoms
    M = dense_M(pix, W)
    D = (w[:, None] * np.abs(M) ** 2).sum(0)
    for i in range(5):
        k = out["sel"][i]
        d = out["dc"][i] / gam
        if mirror(k, W) != k:
            assert e[i + 1] - e[i] <= -4 * gam * (1 - gam) * abs(d) ** 2 * D[k] + 1e-12 * e[0]


def test_pairs_identity_measurement_recovers_real_sparse_and_equals_two_single_steps():
    W = 8
    pix = [[(e, g)] for e in range(W) for g in range(W)]
    w = np.ones(W * W)
    r0 = rng(92)
    ks = [9, 18, 43]                                        # none self-conjugate
    coef = r0.uniform(0.5, 2.0, 3) * np.exp(2j * np.pi * r0.random(3))
    k1, k2 = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    img = np.zeros((W, W), complex)
    truth = np.zeros(W * W, complex)
    for k, a in zip(ks, coef):
        for kk, aa in ((k, a), (mirror(k, W), np.conj(a))):
            img += aa * np.exp(2j * np.pi * ((kk // W) * k1 + (kk % W) * k2) / W)
            truth[kk] += aa
    y = img.real.ravel()
    p3 = oracle.Params(window=W, nu_max=3, gamma_odc=1.0, q_mode=1, pairs=1)
    out = oracle.window_solve(pix, w, y, p3)
    np.testing.assert_allclose(out["c"].ravel(), truth, atol=1e-12)
    F = np.fft.fft2(img.real).ravel()
    kstar = int(np.argmax(np.abs(F)))
    kstar = min(kstar, mirror(kstar, W))
    assert out["sel"][0] == kstar
    np.testing.assert_allclose(out["dc"][0], F[kstar] / W ** 2, rtol=1e-12)
    # orthogonal atoms: one pair step == the two single steps k, -k
    single = oracle.window_solve(pix, w, y, oracle.Params(window=W, nu_max=6, gamma_odc=1.0, q_mode=1))
    np.testing.assert_allclose(single["c"], out["c"], atol=1e-12)


def test_pairs_direct_equals_recurrent_w16_full_image():
    f, mask, y = synth.workload("rljsde_64x64")
    p = oracle.Params(window=16, nu_max=40, pairs=1)
    a, ta = oracle.reconstruct(y, mask, p, trace=True)
    b, tb = oracle.reconstruct(y, mask, p, recurrent=True, trace=True)
    assert (ta["sel"] == tb["sel"]).all()
    assert np.max(np.abs(a - b)) <= 1e-10
